// C-ABI of libpolybin: context, host planner (bin table, pruned boxes, triplets, P_ell mode lists) and the
// pipelines that chain the kernels of fft.cuh and contract.cuh.  See include/polybin.h for the contract.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "common.cuh"
#include "contract.cuh"
#include "fft.cuh"
#include "polybin.h"
#include "polybin_internal.h"

namespace pb {

static thread_local std::string g_init_error;

int fail(polybin_ctx* ctx, int status, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (ctx) ctx->err = buf; else g_init_error = buf;
    return status;
}

int fail_cuda(polybin_ctx* ctx, cudaError_t e, const char* what, const char* file, int line) {
    return fail(ctx, e == cudaErrorMemoryAllocation ? POLYBIN_ENOMEM : POLYBIN_ECUDA, "%s failed: %s (%s:%d)", what,
                cudaGetErrorString(e), file, line);
}

static AxisRange axis_box(int m, int n) {
    AxisRange r;
    if (2 * m + 1 <= n) { r.lo = -m; r.cnt = 2 * m + 1; }
    else { r.lo = -n / 2; r.cnt = n; }
    return r;
}

static AxisRange z_box(int m, int n) {
    AxisRange r;
    r.lo = 0;
    r.cnt = std::min(m, n / 2) + 1;
    return r;
}

// Largest integer f >= 0 with kf * sqrt(f*f) < e (the same float64 expression as the bin table).
static int max_component(double kf, double e) {
    int f = 0;
    while (kf * std::sqrt((double)(f + 1) * (f + 1)) < e) ++f;
    return f;
}

template <typename T>
static int set_smem(polybin_ctx* ctx, const void* fn, size_t bytes) {
    if (bytes > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        if (e != cudaSuccess) return fail_cuda(ctx, e, "cudaFuncSetAttribute", __FILE__, __LINE__);
    }
    return POLYBIN_OK;
}

static int launch_check(polybin_ctx* ctx, const char* what) {
    ctx->launches += 1;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail_cuda(ctx, e, what, __FILE__, __LINE__);
    return POLYBIN_OK;
}

// Lines per CTA of the z-passes and columns per CTA of the strided passes (the kernels' compile-time choice).
template <typename T> static int lines_per_cta(int n) { return lines_per_cta_of<T>(n); }
template <typename T> static int cols_per_cta(int n) { return cols_per_cta_of<T>(n); }

template <typename T> static const C<T>* twiddles(polybin_ctx* ctx, int axis);
template <> const float2* twiddles<float>(polybin_ctx* ctx, int axis) { return (const float2*)ctx->d_tw_f[axis]; }
template <> const double2* twiddles<double>(polybin_ctx* ctx, int axis) { return (const double2*)ctx->d_tw_d[axis]; }

// ----------------------------------------------------------------------------------------------- pipelines

// a1: pruned forward transform of one real field on grid ig (optionally times m1 * m2) into the box of the wave
// numbers |n_i| <= m (the same box on every grid with more than 2m points per axis).
template <typename T, typename TIN, typename TM>
int run_forward(polybin_ctx* ctx, const TIN* in, const TM* m1, const TM* m2, C<T>* t1, C<T>* t2, C<T>* box,
                const InvGrid& ig) {
    const int N0 = ig.N[0], N1 = ig.N[1], N2 = ig.N[2];
    const int Bz = ctx->gz.cnt, By = ctx->gy.cnt;
    const long nlines = (long)N0 * N1;
    auto tw = [&](int a) { return (const C<T>*)(sizeof(T) == 4 ? ig.tw_f[a] : ig.tw_d[a]); };
    int rc = POLYBIN_OK;
    StageTimer timer(ctx, kStageForward);
    {
        const int LP = lines_per_cta<T>(N2);
        const size_t sm = (2 * (size_t)N2 * (LP + 1) + N2) * sizeof(C<T>);
        const unsigned nblk = (unsigned)((nlines + 2 * LP - 1) / (2 * LP));
        PB_WITH_NT(N2, NT, {
            if ((rc = set_smem<T>(ctx, (const void*)k_fwd_z<T, TIN, TM, NT>, sm))) return rc;
            k_fwd_z<T, TIN, TM, NT><<<nblk, 256, sm, ctx->stream>>>(in, m1, m2, t1, nlines, Bz, ig.plan[2], tw(2), LP);
        })
        if ((rc = launch_check(ctx, "k_fwd_z"))) return rc;
    }
    {
        const int TK = cols_per_cta<T>(N1);
        const size_t sm = (2 * (size_t)N1 * TK + N1) * sizeof(C<T>);
        ColBatch b;
        ColItem& it = b.it[0];
        it.in = t1; it.out = t2;
        it.in_os = (long)N1 * Bz; it.in_es = Bz; it.out_os = (long)By * Bz; it.out_es = Bz;
        it.ncols = Bz; it.nouter = N0; it.rng = ctx->gy;
        dim3 grid((Bz + TK - 1) / TK, N0, 1);
        PB_WITH_NT(N1, NT, {
            if ((rc = set_smem<T>(ctx, (const void*)k_col<T, -1, NT>, sm))) return rc;
            k_col<T, -1, NT><<<grid, 256, sm, ctx->stream>>>(b, ig.plan[1], tw(1), TK);
        })
        if ((rc = launch_check(ctx, "k_col fwd y"))) return rc;
    }
    {
        const int TK = cols_per_cta<T>(N0);
        const size_t sm = (2 * (size_t)N0 * TK + N0) * sizeof(C<T>);
        ColBatch b;
        ColItem& it = b.it[0];
        const int ncols = By * Bz;
        it.in = t2; it.out = box;
        it.in_os = 0; it.in_es = ncols; it.out_os = 0; it.out_es = ncols;
        it.ncols = ncols; it.nouter = 1; it.rng = ctx->gx;
        dim3 grid((ncols + TK - 1) / TK, 1, 1);
        PB_WITH_NT(N0, NT, {
            if ((rc = set_smem<T>(ctx, (const void*)k_col<T, -1, NT>, sm))) return rc;
            k_col<T, -1, NT><<<grid, 256, sm, ctx->stream>>>(b, ig.plan[0], tw(0), TK);
        })
        if ((rc = launch_check(ctx, "k_col fwd x"))) return rc;
    }
    return POLYBIN_OK;
}

template <typename T, typename TIN, typename TM>
int run_forward(polybin_ctx* ctx, const TIN* in, const TM* m1, const TM* m2, C<T>* t1, C<T>* t2, C<T>* box) {
    return run_forward<T, TIN, TM>(ctx, in, m1, m2, t1, t2, box, ctx->fg);
}

// a2: shell maps g_b = IFT[Theta_b L_ell D] for all bins on grid ig (box == nullptr: unit spectrum, giving t_b).
// The inverse DFT is normalised by the data grid's 1/N on either grid, so a map on the contraction grid holds the
// same band-limited function as on the data grid, sampled at fewer points.
template <typename T>
int run_shells(polybin_ctx* ctx, const C<T>* box, C<T>* u1, C<T>* u2, T* g, int ell, const InvGrid& ig) {
    return run_shells_m<T>(ctx, box, u1, u2, g, ell, kLegendreM, ig);
}

template <typename T>
int run_shells_m(polybin_ctx* ctx, const C<T>* box, C<T>* u1, C<T>* u2, T* g, int ell, int m, const InvGrid& ig) {
    const int N0 = ig.N[0], N1 = ig.N[1], N2 = ig.N[2];
    const int nb = ctx->nb;
    int rc = POLYBIN_OK;
    auto tw = [&](int a) { return (const C<T>*)(sizeof(T) == 4 ? ig.tw_f[a] : ig.tw_d[a]); };
    StageTimer timer(ctx, kStageShells);
    {
        const int TK = cols_per_cta<T>(N0);
        const size_t sm = (2 * (size_t)N0 * TK + N0) * sizeof(C<T>);
        XInvBatch b;
        int maxcols = 0;
        for (int i = 0; i < nb; ++i) {
            const BinBox& bb = ig.bbox[i];
            b.it[i].out = u1 + bb.u1_off;
            b.it[i].rx = bb.rx; b.it[i].ry = bb.ry; b.it[i].rz = bb.rz;
            b.it[i].bin = i;
            b.it[i].slo = ctx->bin_slo[i];
            b.it[i].shi = ctx->bin_shi[i];
            b.it[i].ell = ell;
            b.it[i].m = m;
            maxcols = std::max(maxcols, bb.ry.cnt * bb.rz.cnt);
        }
        if (N0 == 288 && sizeof(T) == 4) {
            // register-resident 288-point x lines, 16 columns of the bin's box a CTA
            dim3 grid288((maxcols + kY288Cols - 1) / kY288Cols, nb, 1);
            k_inv_x288_filter<<<grid288, kY288Threads, y288_smem(), ctx->stream>>>(
                b, (const float2*)box, ctx->gx, ctx->gy, ctx->gz, (float)(1.0 / (double)ctx->ncell), (const float2*)tw(0));
        } else {
            dim3 grid((maxcols + TK - 1) / TK, nb, 1);
            PB_WITH_NT_INV(N0, NT, {
                if ((rc = set_smem<T>(ctx, (const void*)k_inv_x_filter<T, NT>, sm))) return rc;
                k_inv_x_filter<T, NT><<<grid, 256, sm, ctx->stream>>>(b, box, ctx->gx, ctx->gy, ctx->gz,
                                                                      T(1.0 / (double)ctx->ncell), ig.plan[0], tw(0), TK);
            })
        }
        if ((rc = launch_check(ctx, "k_inv_x_filter"))) return rc;
    }
    {
        const int TK = cols_per_cta<T>(N1);
        const size_t sm = (2 * (size_t)N1 * TK + N1) * sizeof(C<T>);
        ColBatch b;
        int maxc = 0;
        for (int i = 0; i < nb; ++i) {
            const BinBox& bb = ig.bbox[i];
            ColItem& it = b.it[i];
            it.in = u1 + bb.u1_off; it.out = u2 + bb.u2_off;
            it.in_os = (long)bb.ry.cnt * bb.rz.cnt; it.in_es = bb.rz.cnt;
            it.out_os = (long)N1 * bb.rz.cnt; it.out_es = bb.rz.cnt;
            it.ncols = bb.rz.cnt; it.nouter = N0; it.rng = bb.ry;
            maxc = std::max(maxc, bb.rz.cnt);
        }
        if (N1 == 288 && sizeof(T) == 4) {
            // register-resident 288-point columns, 16 wave numbers kz a CTA
            dim3 grid288((maxc + kY288Cols - 1) / kY288Cols, N0, nb);
            k_inv_y288<<<grid288, kY288Threads, y288_smem(), ctx->stream>>>(b, (const float2*)tw(1));
        } else {
            dim3 grid((maxc + TK - 1) / TK, N0, nb);
            PB_WITH_NT_INV(N1, NT, {
                if ((rc = set_smem<T>(ctx, (const void*)k_col<T, +1, NT>, sm))) return rc;
                k_col<T, +1, NT><<<grid, 256, sm, ctx->stream>>>(b, ig.plan[1], tw(1), TK);
            })
        }
        if ((rc = launch_check(ctx, "k_col inv y"))) return rc;
    }
    {
        const int LP = lines_per_cta<T>(N2);
        const size_t sm = (2 * (size_t)N2 * (LP + 1) + N2) * sizeof(C<T>);
        ZInvBatch b;
        for (int i = 0; i < nb; ++i) {
            const BinBox& bb = ig.bbox[i];
            b.it[i].in = u2 + bb.u2_off;
            b.it[i].out = g + (size_t)i * ig.ncell;
            b.it[i].kin = bb.rz.cnt;
        }
        const long nlines = (long)N0 * N1;
        if (N2 == 512) {
            // register-resident 512-point transform, 16 line pairs per CTA
            const int lpc = 16;
            dim3 grid512((unsigned)(((nlines + 1) / 2 + lpc - 1) / lpc), nb, 1);
            k_inv_z512<T><<<grid512, 256, 0, ctx->stream>>>(b, nlines, T(1), (const T*)nullptr, tw(2), lpc);
        } else if (N2 == 256) {
            // register-resident 256-point transform, one warp a line pair, 16 line pairs per CTA
            const int lpc = 16;
            dim3 grid256((unsigned)(((nlines + 1) / 2 + lpc - 1) / lpc), nb, 1);
            k_inv_z256<T><<<grid256, 256, 0, ctx->stream>>>(b, nlines, T(1), (const T*)nullptr, tw(2), lpc);
        } else if (N2 == 288 && sizeof(T) == 4) {
            // register-resident 288-point transform, 128 line pairs per CTA (8 rounds of 16, each round's input
            // staged one round ahead by one bulk copy of the TMA engine; a copy that never lands raises the
            // staging error flag, reported at the next read of the flags)
            if ((rc = ensure_err_flag(ctx))) return rc;
            const int ppc = 128;
            int kin_max = 1;
            for (int i = 0; i < nb; ++i) kin_max = std::max(kin_max, b.it[i].kin);
            const size_t smz = z288_smem(kin_max);
            dim3 grid288((unsigned)(((nlines + 1) / 2 + ppc - 1) / ppc), nb, 1);
            if ((rc = set_smem<T>(ctx, (const void*)k_inv_z288, smz))) return rc;
            k_inv_z288<<<grid288, kZ288Threads, smz, ctx->stream>>>(b, nlines, 1.f, (const float*)nullptr,
                                                                    (const float2*)tw(2), ppc,
                                                                    ctx->d_err + kErrStaging);
        } else {
            dim3 grid((unsigned)((nlines + 2 * LP - 1) / (2 * LP)), nb, 1);
            PB_WITH_NT_INV(N2, NT, {
                if ((rc = set_smem<T>(ctx, (const void*)k_inv_z<T, NT>, sm))) return rc;
                k_inv_z<T, NT><<<grid, 256, sm, ctx->stream>>>(b, nlines, T(1), (const T*)nullptr, ig.plan[2], tw(2), LP);
            })
        }
        if ((rc = launch_check(ctx, "k_inv_z"))) return rc;
    }
    return POLYBIN_OK;
}

// Launches the staging-wait self-test into the staging error flag (the caller clears and reads it).
int run_bulk_wait_selftest(polybin_ctx* ctx, unsigned limit) {
    k_bulk_wait_selftest<<<1, 32, 0, ctx->stream>>>(ctx->d_err + kErrStaging, limit);
    return launch_check(ctx, "k_bulk_wait_selftest");
}

ContractGeom contract_geom(int nb, int nh, long ncell) {
    ContractGeom G;
    G.nb = nb; G.nh = nh; G.npairs = nb * (nb + 1) / 2;
    G.ct = (nh + kTN - 1) / kTN;
    G.rt = 256 / G.ct;
    const int need = (G.npairs + kTM - 1) / kTM * kTM;
    G.rows_cta = std::min(G.rt * kTM, need);
    G.nhp = G.ct * kTN;
    G.ngroups = (G.npairs + G.rows_cta - 1) / G.rows_cta;
    const long nchunks = (ncell + kCH - 1) / kCH;
    long ncb = std::max(1L, std::min(nchunks, (long)(4 * 152 / G.ngroups)));
    G.cells_cta = ((ncell + ncb - 1) / ncb + kCH - 1) / kCH * kCH;
    G.ncb = (int)((ncell + G.cells_cta - 1) / G.cells_cta);
    return G;
}

// a3: contraction; result (device, [npairs][nh] doubles) in d_out.
template <typename T>
int run_contract(polybin_ctx* ctx, const T* g, int ng, const T* h, int nh, double* d_partial, size_t partial_cap,
                 double* d_out, long ncell) {
    int rc;
    StageTimer timer(ctx, kStageContract);
    ContractGeom G = contract_geom(ng, nh, ncell);
    if ((size_t)G.ncb * G.npairs * G.nh > partial_cap) return fail(ctx, POLYBIN_EINVAL, "contract: partial buffer too small");
    const size_t sm = ((size_t)kCH * G.rows_cta + (size_t)kCH * G.nhp + (size_t)ng * (kCH + 1)) * sizeof(T) + 16;
    if ((rc = set_smem<T>(ctx, (const void*)k_contract<T>, sm))) return rc;
    dim3 grid(G.ngroups, G.ncb, 1);
    k_contract<T><<<grid, 256, sm, ctx->stream>>>(g, h, ncell, ctx->d_pairs + pairs_offset(ng), G, d_partial);
    if ((rc = launch_check(ctx, "k_contract"))) return rc;
    const long nout = (long)G.npairs * G.nh;
    k_reduce_partials<<<(unsigned)((nout + 255) / 256), 256, 0, ctx->stream>>>(d_partial, G.ncb, nout, d_out);
    return launch_check(ctx, "k_reduce_partials");
}

// a4: P_ell binning partials [nb][nseg][nell] (device, ctx->d_pkpart) from the box spectrum.
template <typename T>
int run_pkbin_dev(polybin_ctx* ctx, const C<T>* box) {
    StageTimer timer(ctx, kStagePk);
    k_pk_bin<T><<<dim3(ctx->nb, ctx->pk_nseg, 1), 256, 0, ctx->stream>>>(box, ctx->d_offs, ctx->d_coef, ctx->nmodes,
                                                                         ctx->d_bin_start, ctx->nell, ctx->pk_seg_len,
                                                                         ctx->d_pkpart);
    return launch_check(ctx, "k_pk_bin");
}

// a4: P_ell numerators num[ell][b] (host) from the box spectrum (segments summed in order on the host).
template <typename T>
int run_pkbin(polybin_ctx* ctx, const C<T>* box, std::vector<double>& num) {
    int rc;
    const int nb = ctx->nb, nell = ctx->nell;
    if ((rc = run_pkbin_dev<T>(ctx, box))) return rc;
    std::vector<double> part((size_t)nb * ctx->pk_nseg * nell);
    PB_CUDA_OK(cudaMemcpyAsync(part.data(), ctx->d_pkpart, part.size() * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    PB_CUDA_OK(cudaStreamSynchronize(ctx->stream));
    num.assign((size_t)nell * nb, 0.0);
    for (int b = 0; b < nb; ++b)
        for (int s = 0; s < ctx->pk_nseg; ++s)
            for (int l = 0; l < nell; ++l) num[(size_t)l * nb + b] += part[((size_t)b * ctx->pk_nseg + s) * nell + l];
    return POLYBIN_OK;
}

template int run_forward<float, float, float>(polybin_ctx*, const float*, const float*, const float*, float2*, float2*, float2*);
template int run_forward<float, float, float>(polybin_ctx*, const float*, const float*, const float*, float2*, float2*,
                                              float2*, const InvGrid&);
template int run_forward<double, double, double>(polybin_ctx*, const double*, const double*, const double*, double2*,
                                                 double2*, double2*, const InvGrid&);
template int run_forward<double, float, float>(polybin_ctx*, const float*, const float*, const float*, double2*, double2*, double2*);
template int run_forward<double, double, double>(polybin_ctx*, const double*, const double*, const double*, double2*, double2*, double2*);
template int run_forward<double, double, float>(polybin_ctx*, const double*, const float*, const float*, double2*, double2*, double2*);
template int run_pkbin<float>(polybin_ctx*, const float2*, std::vector<double>&);
template int run_pkbin<double>(polybin_ctx*, const double2*, std::vector<double>&);
template int run_pkbin_dev<float>(polybin_ctx*, const float2*);
template int run_pkbin_dev<double>(polybin_ctx*, const double2*);
template int run_shells<float>(polybin_ctx*, const float2*, float2*, float2*, float*, int, const InvGrid&);
template int run_shells<double>(polybin_ctx*, const double2*, double2*, double2*, double*, int, const InvGrid&);
template int run_shells_m<float>(polybin_ctx*, const float2*, float2*, float2*, float*, int, int, const InvGrid&);
template int run_shells_m<double>(polybin_ctx*, const double2*, double2*, double2*, double*, int, int, const InvGrid&);
template int run_contract<float>(polybin_ctx*, const float*, int, const float*, int, double*, size_t, double*, long);
template int run_contract<double>(polybin_ctx*, const double*, int, const double*, int, double*, size_t, double*, long);

template <>
int run_contract_any<double>(polybin_ctx* ctx, const double* g, int ng, const double* h, int nh, double* part,
                             size_t cap, double* out, long ncell) {
    return run_contract<double>(ctx, g, ng, h, nh, part, cap, out, ncell);
}

// ----------------------------------------------------------------------------------------------- planner

// Smallest even length >= need that make_plan accepts (factors 2, 3, 5; <= 1024), or 0 if there is none.
static int fft_len_at_least(int need) {
    for (int n = std::max(need, 2); n <= 1024; ++n) {
        FftPlan p;
        if (n % 2 == 0 && make_plan(n, p)) return n;
    }
    return 0;
}

// Bin boxes and intermediate offsets of the inverse transforms on grid ig (lengths set by the caller).
static void plan_inv_grid(polybin_ctx* ctx, InvGrid& ig) {
    const int nb = ctx->nb;
    ig.ncell = (long)ig.N[0] * ig.N[1] * ig.N[2];
    for (int a = 0; a < 3; ++a) make_plan(ig.N[a], ig.plan[a]);
    ig.bbox.resize(nb);
    long u1 = 0, u2 = 0;
    for (int b = 0; b < nb; ++b) {
        BinBox& bb = ig.bbox[b];
        const int mb = max_component(ctx->kf, ctx->edges[b + 1]);
        bb.rx = axis_box(mb, ig.N[0]);
        bb.ry = axis_box(mb, ig.N[1]);
        bb.rz = z_box(mb, ig.N[2]);
        bb.u1_off = u1;
        bb.u2_off = u2;
        u1 += (long)ig.N[0] * bb.ry.cnt * bb.rz.cnt;
        u2 += (long)ig.N[0] * ig.N[1] * bb.rz.cnt;
    }
    ig.u1_total = u1;
    ig.u2_total = u2;
}

static int plan_bins(polybin_ctx* ctx) {
    const int nb = ctx->nb;
    const double kf = ctx->kf;
    const double elast = ctx->edges[nb];
    // bin table over integer |n|^2
    const long smax_grid = (long)(ctx->N[0] / 2) * (ctx->N[0] / 2) + (long)(ctx->N[1] / 2) * (ctx->N[1] / 2) +
                           (long)(ctx->N[2] / 2) * (ctx->N[2] / 2);
    long smax = 0;
    while (smax + 1 <= smax_grid && kf * std::sqrt((double)(smax + 1)) < elast) ++smax;
    ctx->smax = (int)smax;
    ctx->lut.assign(smax + 1, (int16_t)-1);
    for (long s = 1; s <= smax; ++s) {
        const double k = kf * std::sqrt((double)s);
        for (int b = 0; b < nb; ++b)
            if (k >= ctx->edges[b] && k < ctx->edges[b + 1]) { ctx->lut[s] = (int16_t)b; break; }
    }
    // each bin is one contiguous range of |n|^2 (ascending edges): the shell filter tests the range, not the table
    ctx->bin_slo.assign(nb, 1);
    ctx->bin_shi.assign(nb, 0);
    for (long s = 1; s <= smax; ++s) {
        const int b = ctx->lut[s];
        if (b < 0) continue;
        if (ctx->bin_shi[b] < ctx->bin_slo[b]) ctx->bin_slo[b] = (int)s;
        ctx->bin_shi[b] = (int)s;
    }
    for (int b = 0; b < nb; ++b)
        for (int s = ctx->bin_slo[b]; s <= ctx->bin_shi[b]; ++s)
            if (ctx->lut[s] != b) return fail(ctx, POLYBIN_EINVAL, "bin %d is not one range of |n|^2", b);
    const int m = max_component(kf, elast);
    ctx->gx = axis_box(m, ctx->N[0]);
    ctx->gy = axis_box(m, ctx->N[1]);
    ctx->gz = z_box(m, ctx->N[2]);
    // Data grid.
    for (int a = 0; a < 3; ++a) ctx->fg.N[a] = ctx->N[a];
    plan_inv_grid(ctx, ctx->fg);
    // Contraction grid.  Every shell map has wave numbers |n_i| <= m on each axis, so a product of three has
    // |n_i| <= 3m, and the sum over the cells of a grid of length L_i per axis picks up exactly the zero mode of that
    // product when L_i > 3m (no nonzero multiple of L_i lies within the product's band).  The data grid sum
    // (when itself alias-free, N_i > 3m) therefore equals (N / N') times the same sum over any grid N' with
    // N'_i > 3m: the triplet sums are evaluated on the smallest such 2-3-5 grid.  Where N_i <= 3m (triangles that
    // wrap around the data grid are part of the sum) the axis keeps its data length.
    for (int a = 0; a < 3; ++a) {
        const int need = 3 * std::min(m, ctx->N[a] / 2) + 1;
        const int L = fft_len_at_least(need);
        ctx->cg.N[a] = (need < ctx->N[a] && L > 0 && L < ctx->N[a]) ? L : ctx->N[a];
    }
    plan_inv_grid(ctx, ctx->cg);
    ctx->cg_ratio = (double)ctx->ncell / (double)ctx->cg.ncell;
    return POLYBIN_OK;
}

static double leg(int ell, double mu2) {
    if (ell == 0) return 1.0;
    if (ell == 2) return 0.5 * (3.0 * mu2 - 1.0);
    return (35.0 * mu2 * mu2 - 30.0 * mu2 + 3.0) / 8.0;
}

static int plan_pk(polybin_ctx* ctx) {
    const int nb = ctx->nb, nell = ctx->nell;
    const int Bx = ctx->gx.cnt, By = ctx->gy.cnt, Bz = ctx->gz.cnt;
    std::vector<std::vector<int>> offs(nb);
    std::vector<std::vector<double>> coef(nb);
    ctx->counts.assign(nb, 0.0);
    ctx->fish_disc.assign((size_t)nb * nell * nell, 0.0);
    for (int ix = 0; ix < Bx; ++ix)
        for (int iy = 0; iy < By; ++iy)
            for (int iz = 0; iz < Bz; ++iz) {
                const long fx = ctx->gx.lo + ix, fy = ctx->gy.lo + iy, fz = iz;
                const long s = fx * fx + fy * fy + fz * fz;
                if (s > ctx->smax) continue;
                const int b = ctx->lut[s];
                if (b < 0) continue;
                const double w = (fz == 0 || 2 * fz == ctx->N[2]) ? 1.0 : 2.0;
                const double mu2 = (double)(fz * fz) / (double)s;
                offs[b].push_back((ix * By + iy) * Bz + iz);
                double L[3];
                for (int l = 0; l < nell; ++l) { L[l] = leg(2 * l, mu2); coef[b].push_back(w * L[l]); }
                ctx->counts[b] += w;
                for (int l = 0; l < nell; ++l)
                    for (int l2 = 0; l2 < nell; ++l2) ctx->fish_disc[((size_t)b * nell + l) * nell + l2] += 0.5 * w * L[l] * L[l2];
            }
    std::vector<int> all_offs, start(nb + 1, 0);
    for (int b = 0; b < nb; ++b) { start[b + 1] = start[b] + (int)offs[b].size(); }
    const long M = start[nb];
    ctx->nmodes = M;
    std::vector<double> all_coef((size_t)nell * std::max(M, 1L));
    all_offs.reserve(M);
    for (int b = 0; b < nb; ++b) {
        for (size_t q = 0; q < offs[b].size(); ++q) {
            const long m = start[b] + (long)q;
            all_offs.push_back(offs[b][q]);
            for (int l = 0; l < nell; ++l) all_coef[(size_t)l * M + m] = coef[b][q * nell + l];
        }
    }
    long maxlen = 1;
    for (int b = 0; b < nb; ++b) maxlen = std::max(maxlen, (long)offs[b].size());
    ctx->pk_seg_len = 8192;
    ctx->pk_nseg = (int)((maxlen + ctx->pk_seg_len - 1) / ctx->pk_seg_len);
    polybin_ctx* c = ctx;
    PB_CUDA_OK_C(cudaMalloc(&c->d_offs, sizeof(int) * std::max(M, 1L)));
    PB_CUDA_OK_C(cudaMalloc(&c->d_coef, sizeof(double) * all_coef.size()));
    PB_CUDA_OK_C(cudaMalloc(&c->d_bin_start, sizeof(int) * (nb + 1)));
    PB_CUDA_OK_C(cudaMalloc(&c->d_pkpart, sizeof(double) * (size_t)nb * c->pk_nseg * nell));
    PB_CUDA_OK_C(cudaMalloc(&c->d_pkout, sizeof(double) * (size_t)nb * nell));
    PB_CUDA_OK_C(cudaMalloc(&c->d_counts, sizeof(double) * nb));
    PB_CUDA_OK_C(cudaMemcpy(c->d_counts, c->counts.data(), sizeof(double) * nb, cudaMemcpyHostToDevice));
    if (M) PB_CUDA_OK_C(cudaMemcpy(c->d_offs, all_offs.data(), sizeof(int) * M, cudaMemcpyHostToDevice));
    PB_CUDA_OK_C(cudaMemcpy(c->d_coef, all_coef.data(), sizeof(double) * all_coef.size(), cudaMemcpyHostToDevice));
    PB_CUDA_OK_C(cudaMemcpy(c->d_bin_start, start.data(), sizeof(int) * (nb + 1), cudaMemcpyHostToDevice));
    return POLYBIN_OK;
}

// e^{-2 pi i m / n}, m = 0 .. n-1, in float and double (device arrays owned by the caller).
static int make_twiddles(polybin_ctx* ctx, int n, void** f, void** d) {
    std::vector<float2> tf(n);
    std::vector<double2> td(n);
    for (int m = 0; m < n; ++m) {
        const double ang = 2.0 * M_PI * (double)m / (double)n;
        const double cr = std::cos(ang), si = -std::sin(ang);
        td[m] = make_double2(cr, si);
        tf[m] = make_float2((float)cr, (float)si);
    }
    PB_CUDA_OK_C(cudaMalloc(f, sizeof(float2) * n));
    PB_CUDA_OK_C(cudaMalloc(d, sizeof(double2) * n));
    PB_CUDA_OK_C(cudaMemcpy(*f, tf.data(), sizeof(float2) * n, cudaMemcpyHostToDevice));
    PB_CUDA_OK_C(cudaMemcpy(*d, td.data(), sizeof(double2) * n, cudaMemcpyHostToDevice));
    return POLYBIN_OK;
}

static int upload_twiddles(polybin_ctx* ctx) {
    int rc;
    for (int a = 0; a < 3; ++a) {
        if ((rc = make_twiddles(ctx, ctx->N[a], &ctx->d_tw_f[a], &ctx->d_tw_d[a]))) return rc;
        ctx->fg.tw_f[a] = ctx->d_tw_f[a];
        ctx->fg.tw_d[a] = ctx->d_tw_d[a];
        if (ctx->cg.N[a] == ctx->N[a]) {
            ctx->cg.tw_f[a] = ctx->d_tw_f[a];
            ctx->cg.tw_d[a] = ctx->d_tw_d[a];
        } else {
            if ((rc = make_twiddles(ctx, ctx->cg.N[a], &ctx->d_ctw[2 * a], &ctx->d_ctw[2 * a + 1]))) return rc;
            ctx->cg.tw_f[a] = ctx->d_ctw[2 * a];
            ctx->cg.tw_d[a] = ctx->d_ctw[2 * a + 1];
        }
    }
    return POLYBIN_OK;
}

template <typename T>
int alloc_work(polybin_ctx* ctx, Work& w) {
    const long N0 = ctx->N[0], N1 = ctx->N[1];
    const long Bx = ctx->gx.cnt, By = ctx->gy.cnt, Bz = ctx->gz.cnt;
    polybin_ctx* c = ctx;
    w.elem = sizeof(T);
    PB_CUDA_OK_C(cudaMalloc(&w.t1, sizeof(C<T>) * N0 * N1 * Bz));
    PB_CUDA_OK_C(cudaMalloc(&w.t2, sizeof(C<T>) * N0 * By * Bz));
    PB_CUDA_OK_C(cudaMalloc(&w.box, sizeof(C<T>) * Bx * By * Bz));
    PB_CUDA_OK_C(cudaMalloc(&w.u1, sizeof(C<T>) * ctx->cg.u1_total));
    PB_CUDA_OK_C(cudaMalloc(&w.u2, sizeof(C<T>) * ctx->cg.u2_total));
    PB_CUDA_OK_C(cudaMalloc(&w.g, sizeof(T) * (size_t)ctx->nb * ctx->cg.ncell));
    const int np = 64 * 65 / 2;
    ContractGeom G = contract_geom(std::max(ctx->nb, 1), std::max(ctx->nb, 1), ctx->ncell);
    w.partial_cap = (size_t)G.ncb * G.npairs * G.nh;
    // room for any (n_g, n_h <= 64) contraction launched through polybin_contract
    ContractGeom G2 = contract_geom(64, 64, ctx->ncell);
    w.partial_cap = std::max(w.partial_cap, (size_t)G2.ncb * G2.npairs * G2.nh);
    PB_CUDA_OK_C(cudaMalloc(&w.partial, sizeof(double) * w.partial_cap));
    PB_CUDA_OK_C(cudaMalloc(&w.mout, sizeof(double) * (size_t)np * 64));
    return POLYBIN_OK;
}

template <typename T>
int ensure_fine_inv(polybin_ctx* ctx) {
    Work& w = ctx->w;
    if (w.u1f && w.u2f) return POLYBIN_OK;
    PB_CUDA_OK(cudaMalloc(&w.u1f, sizeof(C<T>) * ctx->fg.u1_total));
    PB_CUDA_OK(cudaMalloc(&w.u2f, sizeof(C<T>) * ctx->fg.u2_total));
    return POLYBIN_OK;
}
template int ensure_fine_inv<float>(polybin_ctx*);
template int ensure_fine_inv<double>(polybin_ctx*);

void free_work(Work& w) {
    void* ptrs[] = {w.t1, w.t2, w.box, w.u1, w.u2, w.u1f, w.u2f, w.g, w.g2, w.partial, w.mout};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    w = Work();
}

template int alloc_work<float>(polybin_ctx*, Work&);
template int alloc_work<double>(polybin_ctx*, Work&);

// Host or device input -> device pointer (host data copied into the context's staging buffer).
// Batched input staging.  For host memory and more than one field, field f is copied on the context's copy stream
// into buffer f % 2 while the context stream transforms field f - 1; the context stream waits for the copy, and the
// next copy into a buffer waits until the forward transform that read it has run.  (Pageable memory works too, but
// the driver then copies synchronously and nothing overlaps: pass pinned memory.)
struct InputStager {
    polybin_ctx* ctx;
    const float* base;
    int batch;
    bool on = false;
    int init() {
        cudaPointerAttributes at;
        cudaError_t e = cudaPointerGetAttributes(&at, base);
        if (e != cudaSuccess) { cudaGetLastError(); at.type = cudaMemoryTypeUnregistered; }
        on = batch > 1 && !ctx->capturing && at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged;
        if (!on) return POLYBIN_OK;
        const size_t n = (size_t)ctx->ncell;
        if (n > ctx->stage_cap) {
            for (int i = 0; i < 2; ++i) {
                if (ctx->d_stage[i]) cudaFree(ctx->d_stage[i]);
                ctx->d_stage[i] = nullptr;
            }
            ctx->stage_cap = 0;
            for (int i = 0; i < 2; ++i) PB_CUDA_OK(cudaMalloc(&ctx->d_stage[i], sizeof(float) * n));
            ctx->stage_cap = n;
        }
        if (!ctx->cstream) PB_CUDA_OK(cudaStreamCreateWithFlags(&ctx->cstream, cudaStreamNonBlocking));
        for (int i = 0; i < 2; ++i) {
            if (!ctx->ev_copied[i]) PB_CUDA_OK(cudaEventCreateWithFlags(&ctx->ev_copied[i], cudaEventDisableTiming));
            if (!ctx->ev_used[i]) PB_CUDA_OK(cudaEventCreateWithFlags(&ctx->ev_used[i], cudaEventDisableTiming));
        }
        // the copy stream starts after the work already queued on the context stream
        PB_CUDA_OK(cudaEventRecord(ctx->ev_used[0], ctx->stream));
        PB_CUDA_OK(cudaEventRecord(ctx->ev_used[1], ctx->stream));
        return copy(0);
    }
    int copy(int f) {
        const int s = f & 1;
        PB_CUDA_OK(cudaStreamWaitEvent(ctx->cstream, ctx->ev_used[s], 0));
        PB_CUDA_OK(cudaMemcpyAsync(ctx->d_stage[s], base + (size_t)f * ctx->ncell, sizeof(float) * ctx->ncell,
                                   cudaMemcpyHostToDevice, ctx->cstream));
        PB_CUDA_OK(cudaEventRecord(ctx->ev_copied[s], ctx->cstream));
        return POLYBIN_OK;
    }
    // the device pointer of field f (issuing the copy of field f + 1 first)
    int get(int f, const float** out) {
        if (!on) return resolve_input(ctx, base + (size_t)f * ctx->ncell, ctx->ncell, out);
        int rc;
        if (f + 1 < batch && (rc = copy(f + 1))) return rc;
        PB_CUDA_OK(cudaStreamWaitEvent(ctx->stream, ctx->ev_copied[f & 1], 0));
        *out = ctx->d_stage[f & 1];
        return POLYBIN_OK;
    }
    // field f's buffer has been read (after its forward transform)
    int done(int f) {
        if (on) PB_CUDA_OK(cudaEventRecord(ctx->ev_used[f & 1], ctx->stream));
        return POLYBIN_OK;
    }
};

int resolve_input(polybin_ctx* ctx, const float* p, size_t count, const float** out) {
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) { cudaGetLastError(); at.type = cudaMemoryTypeUnregistered; }
    if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) { *out = p; return POLYBIN_OK; }
    if (count > ctx->in_cap) {
        if (ctx->d_in) cudaFree(ctx->d_in);
        ctx->d_in = nullptr;
        ctx->in_cap = 0;
        PB_CUDA_OK(cudaMalloc(&ctx->d_in, sizeof(float) * count));
        ctx->in_cap = count;
    }
    PB_CUDA_OK(cudaMemcpyAsync(ctx->d_in, p, sizeof(float) * count, cudaMemcpyHostToDevice, ctx->stream));
    *out = ctx->d_in;
    return POLYBIN_OK;
}

// N_abc via the FP64 pipeline on unit fields (cached), evaluated on the contraction grid: T_abc = cg_ratio T'_abc.
int ensure_triplets(polybin_ctx* ctx) {
    if (ctx->trip_ready) return POLYBIN_OK;
    int rc;
    Work tmp;
    Work* w = &ctx->w;
    const bool own = ctx->prec != POLYBIN_FP64;
    if (own) {
        if ((rc = alloc_work_shells_double(ctx, tmp))) { free_work(tmp); return rc; }
        w = &tmp;
    }
    const long cn = ctx->cg.ncell;
    rc = run_shells<double>(ctx, nullptr, (double2*)w->u1, (double2*)w->u2, (double*)w->g, 0, ctx->cg);
    if (!rc) rc = run_contract<double>(ctx, (const double*)w->g, ctx->nb, nullptr, ctx->nb, w->partial, w->partial_cap, w->mout, cn);
    const int nb = ctx->nb, np = nb * (nb + 1) / 2;
    std::vector<double> T((size_t)np * nb);
    if (!rc) {
        cudaError_t e = cudaMemcpyAsync(T.data(), w->mout, sizeof(double) * T.size(), cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) rc = fail_cuda(ctx, e, "N_abc copy", __FILE__, __LINE__);
    }
    if (own) free_work(tmp);
    if (rc) return rc;
    ctx->trip.clear();
    ctx->Tabc.clear();
    ctx->Nabc.clear();
    const double n2 = (double)ctx->ncell * (double)ctx->ncell;
    for (int a = 0; a < nb; ++a)
        for (int b = a; b < nb; ++b)
            for (int c = b; c < nb; ++c) {
                const double t = ctx->cg_ratio * T[(size_t)pair_index(nb, a, b) * nb + c];
                const double cnt = std::nearbyint(n2 * t);
                if (cnt > 0) {
                    ctx->trip.push_back(a); ctx->trip.push_back(b); ctx->trip.push_back(c);
                    ctx->Tabc.push_back(t);
                    ctx->Nabc.push_back(cnt);
                }
            }
    const size_t nt = ctx->Nabc.size();
    std::vector<double> Tv(std::max(nt, (size_t)1), 1.0);
    for (size_t t = 0; t < nt; ++t) Tv[t] = ctx->Tabc[t];
    polybin_ctx* c = ctx;
    PB_CUDA_OK_C(cudaMalloc(&c->d_S, sizeof(double) * Tv.size()));
    PB_CUDA_OK_C(cudaMalloc(&c->d_B, sizeof(double) * Tv.size()));
    PB_CUDA_OK_C(cudaMalloc(&c->d_T, sizeof(double) * Tv.size()));
    PB_CUDA_OK_C(cudaMemcpy(c->d_T, Tv.data(), sizeof(double) * Tv.size(), cudaMemcpyHostToDevice));
    ctx->trip_ready = true;
    // the tensor-core plan is built now, outside any later stream capture
    if (ctx->prec == POLYBIN_SPLIT_TF32X3 && nt > 0 && tc_shape_ok(ctx->cg.ncell, (const float*)ctx->w.g, nb, nullptr, nb))
        return prepare_triplet_tc(ctx);
    return POLYBIN_OK;
}

// FP64 workspace of the N_abc pipeline (unit-field shell maps on the contraction grid and their contraction).
int alloc_work_shells_double(polybin_ctx* ctx, Work& w) {
    polybin_ctx* c = ctx;
    w.elem = sizeof(double);
    PB_CUDA_OK_C(cudaMalloc(&w.u1, sizeof(double2) * ctx->cg.u1_total));
    PB_CUDA_OK_C(cudaMalloc(&w.u2, sizeof(double2) * ctx->cg.u2_total));
    PB_CUDA_OK_C(cudaMalloc(&w.g, sizeof(double) * (size_t)ctx->nb * ctx->cg.ncell));
    ContractGeom G = contract_geom(ctx->nb, ctx->nb, ctx->cg.ncell);
    w.partial_cap = (size_t)G.ncb * G.npairs * G.nh;
    PB_CUDA_OK_C(cudaMalloc(&w.partial, sizeof(double) * w.partial_cap));
    PB_CUDA_OK_C(cudaMalloc(&w.mout, sizeof(double) * (size_t)G.npairs * G.nh));
    return POLYBIN_OK;
}

}  // namespace pb

using namespace pb;

// =============================================================================================== C-ABI

extern "C" int polybin_init(polybin_ctx** out, const int grid[3], const double boxsize[3], const double* k_edges,
                            int n_kbins, int l_max, int prec, void* cuda_stream) {
    if (!out) return fail(nullptr, POLYBIN_EINVAL, "polybin_init: out is NULL");
    *out = nullptr;
    if (!grid || !boxsize || !k_edges) return fail(nullptr, POLYBIN_EINVAL, "polybin_init: NULL argument");
    for (int a = 0; a < 3; ++a) {
        FftPlan p;
        if (grid[a] < 2 || grid[a] % 2 || !make_plan(grid[a], p))
            return fail(nullptr, POLYBIN_EINVAL, "polybin_init: grid[%d] = %d must be even, <= 1024, with factors 2, 3, 5",
                        a, grid[a]);
    }
    if (!(boxsize[0] > 0) || boxsize[0] != boxsize[1] || boxsize[0] != boxsize[2])
        return fail(nullptr, POLYBIN_EINVAL, "polybin_init: the box must be cubic with a positive side");
    if (n_kbins < 1 || n_kbins > kMaxItems) return fail(nullptr, POLYBIN_EINVAL, "polybin_init: 1 <= n_kbins <= 64");
    for (int b = 0; b < n_kbins; ++b)
        if (!(k_edges[b] < k_edges[b + 1]) || !std::isfinite(k_edges[b + 1]) || k_edges[0] < 0)
            return fail(nullptr, POLYBIN_EINVAL, "polybin_init: k_edges must be finite, non-negative and ascending");
    if (l_max < 0 || l_max > 4 || l_max % 2) return fail(nullptr, POLYBIN_EINVAL, "polybin_init: l_max must be 0, 2 or 4");
    if (prec != POLYBIN_FP64 && prec != POLYBIN_FP32 && prec != POLYBIN_SPLIT_TF32X3)
        return fail(nullptr, POLYBIN_EINVAL, "polybin_init: unknown precision %d", prec);
    if (prec == POLYBIN_SPLIT_TF32X3 && !pb::split_tc_available())
        return fail(nullptr, POLYBIN_EINVAL, "polybin_init: the split-TF32 tensor-core contraction is not available");

    polybin_ctx* ctx = new (std::nothrow) polybin_ctx();
    if (!ctx) return fail(nullptr, POLYBIN_ENOMEM, "polybin_init: out of host memory");
    static std::atomic<unsigned long long> next_uid{1};
    ctx->uid = next_uid.fetch_add(1);
    for (int a = 0; a < 3; ++a) ctx->N[a] = grid[a];
    ctx->ncell = (long)grid[0] * grid[1] * grid[2];
    ctx->L = boxsize[0];
    ctx->vol = boxsize[0] * boxsize[1] * boxsize[2];
    ctx->kf = 2.0 * M_PI / boxsize[0];
    ctx->nb = n_kbins;
    ctx->edges.assign(k_edges, k_edges + n_kbins + 1);
    ctx->lmax = l_max;
    ctx->nell = l_max / 2 + 1;
    ctx->prec = prec;
    ctx->stream = (cudaStream_t)cuda_stream;
    for (int a = 0; a < 3; ++a) make_plan(grid[a], ctx->plan[a]);
    int rc = plan_bins(ctx);
    if (!rc) rc = upload_twiddles(ctx);
    if (!rc) {
        cudaError_t e = cudaMalloc(&ctx->d_lut, sizeof(int16_t) * ctx->lut.size());
        if (e == cudaSuccess) e = cudaMemcpy(ctx->d_lut, ctx->lut.data(), sizeof(int16_t) * ctx->lut.size(), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) rc = fail_cuda(ctx, e, "lut upload", __FILE__, __LINE__);
    }
    if (!rc) {
        std::vector<short2> pairs;
        for (int n = 1; n <= 64; ++n)
            for (int j = 0; j < n; ++j)
                for (int k = j; k < n; ++k) pairs.push_back(make_short2((short)j, (short)k));
        cudaError_t e = cudaMalloc(&ctx->d_pairs, sizeof(short2) * pairs.size());
        if (e == cudaSuccess) e = cudaMemcpy(ctx->d_pairs, pairs.data(), sizeof(short2) * pairs.size(), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) rc = fail_cuda(ctx, e, "pairs upload", __FILE__, __LINE__);
    }
    if (!rc) rc = plan_pk(ctx);
    // the device error flags exist from the start (kernels captured into CUDA graphs write them)
    if (!rc) rc = ensure_err_flag(ctx);
    if (!rc) rc = (prec == POLYBIN_FP64) ? alloc_work<double>(ctx, ctx->w) : alloc_work<float>(ctx, ctx->w);
    if (!rc && prec == POLYBIN_SPLIT_TF32X3) rc = tf32_selfcheck(ctx);
    if (rc) {
        g_init_error = ctx->err;
        polybin_destroy(ctx);
        return rc;
    }
    *out = ctx;
    return POLYBIN_OK;
}

extern "C" void polybin_destroy(polybin_ctx* ctx) {
    if (!ctx) return;
    free_work(ctx->w);
    if (ctx->cstream) cudaStreamSynchronize(ctx->cstream);
    void* ptrs[] = {ctx->d_lut, ctx->d_pairs, ctx->d_offs, ctx->d_coef, ctx->d_bin_start, ctx->d_pkpart, ctx->d_in,
                    ctx->d_stage[0], ctx->d_stage[1], ctx->d_pkout, ctx->d_counts,
                    ctx->d_tw_f[0], ctx->d_tw_f[1], ctx->d_tw_f[2], ctx->d_tw_d[0], ctx->d_tw_d[1], ctx->d_tw_d[2],
                    ctx->d_ctw[0], ctx->d_ctw[1], ctx->d_ctw[2], ctx->d_ctw[3], ctx->d_ctw[4], ctx->d_ctw[5]};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    destroy_extras(ctx);
    for (int i = 0; i < 2; ++i) {
        if (ctx->ev_copied[i]) cudaEventDestroy(ctx->ev_copied[i]);
        if (ctx->ev_used[i]) cudaEventDestroy(ctx->ev_used[i]);
    }
    if (ctx->cstream) cudaStreamDestroy(ctx->cstream);
    if (ctx->tev[0]) {
        harvest_stage_times(ctx);
        for (cudaEvent_t ev : ctx->tev) cudaEventDestroy(ev);
    }
    delete ctx;
}

extern "C" const char* polybin_last_error(const polybin_ctx* ctx) {
    return ctx ? ctx->err.c_str() : g_init_error.c_str();
}

extern "C" int polybin_num_triplets(polybin_ctx* ctx, int* n) {
    if (!ctx || !n) return fail(ctx, POLYBIN_EINVAL, "polybin_num_triplets: NULL argument");
    int rc = ensure_triplets(ctx);
    if (rc) return rc;
    *n = (int)ctx->Nabc.size();
    return POLYBIN_OK;
}

extern "C" int polybin_get_triplets(polybin_ctx* ctx, int* abc, double* n_abc) {
    if (!ctx || !abc) return fail(ctx, POLYBIN_EINVAL, "polybin_get_triplets: NULL argument");
    int rc = ensure_triplets(ctx);
    if (rc) return rc;
    std::memcpy(abc, ctx->trip.data(), sizeof(int) * ctx->trip.size());
    if (n_abc) std::memcpy(n_abc, ctx->Nabc.data(), sizeof(double) * ctx->Nabc.size());
    return POLYBIN_OK;
}

// Ideal bispectrum and/or continuous-normalisation P_ell of `batch` fields: per field one forward transform, then
// the P binning and its normalisation (eq. fish-ideal-continuous) and the shell maps, triplet sums and their
// normalisation B = (V^2 / N^3) S / T (Sec. 4.4.1), all on the device; one read-back and one synchronisation per
// field.
template <typename T>
static int bk_pk_t(polybin_ctx* ctx, const float* delta, int batch, double* bk_out, double* pk_out) {
    int rc;
    const int nb = ctx->nb, nell = ctx->nell;
    const size_t nt = ctx->Nabc.size();
    InputStager st{ctx, delta, batch};
    if ((rc = st.init())) return rc;
    for (int f = 0; f < batch; ++f) {
        const float* in;
        if ((rc = st.get(f, &in))) return rc;
        Work& w = ctx->w;
        if ((rc = run_forward<T, float, float>(ctx, in, (const float*)nullptr, (const float*)nullptr, (C<T>*)w.t1, (C<T>*)w.t2, (C<T>*)w.box))) return rc;
        if ((rc = st.done(f))) return rc;
        if (pk_out) {
            if ((rc = run_pkbin_dev<T>(ctx, (const C<T>*)w.box))) return rc;
            if ((rc = run_pk_normalise(ctx, ctx->d_pkout))) return rc;
            PB_CUDA_OK(cudaMemcpyAsync(pk_out + (size_t)f * nell * nb, ctx->d_pkout, sizeof(double) * nell * nb,
                                       cudaMemcpyDeviceToHost, ctx->stream));
        }
        if (bk_out && nt > 0) {
            if ((rc = run_shells<T>(ctx, (const C<T>*)w.box, (C<T>*)w.u1, (C<T>*)w.u2, (T*)w.g, 0, ctx->cg))) return rc;
            if ((rc = run_triplet_sums<T>(ctx, (const T*)w.g, ctx->d_S))) return rc;
            if ((rc = run_bk_normalise(ctx, ctx->d_S, ctx->d_B))) return rc;
            PB_CUDA_OK(cudaMemcpyAsync(bk_out + (size_t)f * nt, ctx->d_B, sizeof(double) * nt, cudaMemcpyDeviceToHost,
                                       ctx->stream));
        }
        PB_CUDA_OK(cudaStreamSynchronize(ctx->stream));
    }
    return POLYBIN_OK;
}

// Bispectrum multipoles ell = 0, 2, .., lmax_b of `batch` fields (Sec. 4.1, eq. ideal-bk): one forward transform,
// the ell = 0 shell maps g and, per ell > 0, the Legendre-weighted maps g_{c,ell} = IFT[Theta_c L_ell D]; the sums
// S^ell_abc = sum_x g_a g_b g_{c,ell} and B_ell = (2 ell + 1) (V^2 / N^3) S^ell / T_abc on the device.
template <typename T>
static int bk_multipoles_t(polybin_ctx* ctx, const float* delta, int batch, int lmax_b, double* bk_out) {
    int rc;
    const size_t nt = ctx->Nabc.size();
    const int nl = lmax_b / 2 + 1;
    Work& w = ctx->w;
    if (lmax_b > 0 && !w.g2) PB_CUDA_OK(cudaMalloc(&w.g2, sizeof(T) * (size_t)ctx->nb * ctx->cg.ncell));
    InputStager st{ctx, delta, batch};
    if ((rc = st.init())) return rc;
    for (int f = 0; f < batch; ++f) {
        const float* in;
        if ((rc = st.get(f, &in))) return rc;
        if ((rc = run_forward<T, float, float>(ctx, in, (const float*)nullptr, (const float*)nullptr, (C<T>*)w.t1, (C<T>*)w.t2, (C<T>*)w.box))) return rc;
        if ((rc = st.done(f))) return rc;
        if (nt == 0) continue;
        if ((rc = run_shells<T>(ctx, (const C<T>*)w.box, (C<T>*)w.u1, (C<T>*)w.u2, (T*)w.g, 0, ctx->cg))) return rc;
        for (int il = 0; il < nl; ++il) {
            const int ell = 2 * il;
            if (ell == 0) {
                if ((rc = run_triplet_sums<T>(ctx, (const T*)w.g, ctx->d_S))) return rc;
            } else {
                if ((rc = run_shells<T>(ctx, (const C<T>*)w.box, (C<T>*)w.u1, (C<T>*)w.u2, (T*)w.g2, ell, ctx->cg))) return rc;
                if ((rc = run_triplet_sums_ell<T>(ctx, (const T*)w.g, (const T*)w.g2, ctx->d_S))) return rc;
            }
            if ((rc = run_bk_normalise(ctx, ctx->d_S, ctx->d_B, 2.0 * ell + 1.0))) return rc;
            PB_CUDA_OK(cudaMemcpyAsync(bk_out + ((size_t)f * nl + il) * nt, ctx->d_B, sizeof(double) * nt,
                                       cudaMemcpyDeviceToHost, ctx->stream));
        }
        PB_CUDA_OK(cudaStreamSynchronize(ctx->stream));
    }
    return POLYBIN_OK;
}

extern "C" int polybin_bk_ideal_multipoles(polybin_ctx* ctx, const float* delta, int batch, int lmax_b, double* bk_out) {
    if (!ctx || !delta || !bk_out || batch < 0 || lmax_b < 0 || lmax_b > 4 || lmax_b % 2)
        return fail(ctx, POLYBIN_EINVAL, "polybin_bk_ideal_multipoles: bad argument (lmax_b must be 0, 2 or 4)");
    int rc = ensure_triplets(ctx);
    if (rc) return rc;
    return ctx->prec == POLYBIN_FP64 ? bk_multipoles_t<double>(ctx, delta, batch, lmax_b, bk_out)
                                     : bk_multipoles_t<float>(ctx, delta, batch, lmax_b, bk_out);
}

extern "C" int polybin_bk_ideal(polybin_ctx* ctx, const float* delta, int batch, double* bk_out) {
    if (!ctx || !delta || !bk_out || batch < 0) return fail(ctx, POLYBIN_EINVAL, "polybin_bk_ideal: bad argument");
    int rc = ensure_triplets(ctx);
    if (rc) return rc;
    return ctx->prec == POLYBIN_FP64 ? bk_pk_t<double>(ctx, delta, batch, bk_out, nullptr)
                                     : bk_pk_t<float>(ctx, delta, batch, bk_out, nullptr);
}

// Discrete-Fisher P_ell (eq. pk-limit): p = F^-1 p_num per bin, p_num = (1/2)(1/N) num, F = (1/2) sum L L' (a 3 x 3
// solve per bin on the host), physical units x V/N.
template <typename T>
static int pk_discrete_t(polybin_ctx* ctx, const float* delta, int batch, double* pk_out) {
    int rc;
    const int nb = ctx->nb, nell = ctx->nell;
    std::vector<double> num;
    for (int f = 0; f < batch; ++f) {
        const float* in;
        if ((rc = resolve_input(ctx, delta + (size_t)f * ctx->ncell, ctx->ncell, &in))) return rc;
        Work& w = ctx->w;
        if ((rc = run_forward<T, float, float>(ctx, in, (const float*)nullptr, (const float*)nullptr, (C<T>*)w.t1, (C<T>*)w.t2, (C<T>*)w.box))) return rc;
        if ((rc = run_pkbin<T>(ctx, (const C<T>*)w.box, num))) return rc;
        double* o = pk_out + (size_t)f * nell * nb;
        const double N = (double)ctx->ncell;
        for (int b = 0; b < nb; ++b) {
            double A[3][4];
            for (int l = 0; l < nell; ++l) {
                for (int l2 = 0; l2 < nell; ++l2) A[l][l2] = ctx->fish_disc[((size_t)b * nell + l) * nell + l2];
                A[l][nell] = 0.5 * num[(size_t)l * nb + b] / N;
            }
            double x[3] = {0, 0, 0};
            if (!solve_small(A, nell, x)) for (int l = 0; l < nell; ++l) x[l] = NAN;
            for (int l = 0; l < nell; ++l) o[(size_t)l * nb + b] = x[l] * ctx->vol / N;
        }
    }
    return POLYBIN_OK;
}

extern "C" int polybin_pk(polybin_ctx* ctx, const float* delta, int batch, double* pk_out) {
    if (!ctx || !delta || !pk_out || batch < 0) return fail(ctx, POLYBIN_EINVAL, "polybin_pk: bad argument");
    return ctx->prec == POLYBIN_FP64 ? bk_pk_t<double>(ctx, delta, batch, nullptr, pk_out)
                                     : bk_pk_t<float>(ctx, delta, batch, nullptr, pk_out);
}

extern "C" int polybin_pk_discrete(polybin_ctx* ctx, const float* delta, int batch, double* pk_out) {
    if (!ctx || !delta || !pk_out || batch < 0) return fail(ctx, POLYBIN_EINVAL, "polybin_pk_discrete: bad argument");
    return ctx->prec == POLYBIN_FP64 ? pk_discrete_t<double>(ctx, delta, batch, pk_out)
                                     : pk_discrete_t<float>(ctx, delta, batch, pk_out);
}

extern "C" int polybin_mode_counts(const polybin_ctx* ctx, double* counts) {
    if (!ctx || !counts) return fail(const_cast<polybin_ctx*>(ctx), POLYBIN_EINVAL, "polybin_mode_counts: NULL argument");
    std::memcpy(counts, ctx->counts.data(), sizeof(double) * ctx->nb);
    return POLYBIN_OK;
}

extern "C" int polybin_spectrum_shape(const polybin_ctx* ctx, int dims[3], int lo[3]) {
    if (!ctx || !dims) return fail(const_cast<polybin_ctx*>(ctx), POLYBIN_EINVAL, "polybin_spectrum_shape: NULL argument");
    dims[0] = ctx->gx.cnt; dims[1] = ctx->gy.cnt; dims[2] = ctx->gz.cnt;
    if (lo) { lo[0] = ctx->gx.lo; lo[1] = ctx->gy.lo; lo[2] = ctx->gz.lo; }
    return POLYBIN_OK;
}

extern "C" int polybin_forward(polybin_ctx* ctx, const float* delta, void* spec_out) {
    if (!ctx || !delta || !spec_out) return fail(ctx, POLYBIN_EINVAL, "polybin_forward: NULL argument");
    int rc;
    Work& w = ctx->w;
    if (ctx->prec == POLYBIN_FP64)
        rc = run_forward<double, float, float>(ctx, delta, (const float*)nullptr, (const float*)nullptr, (double2*)w.t1, (double2*)w.t2, (double2*)spec_out);
    else
        rc = run_forward<float, float, float>(ctx, delta, (const float*)nullptr, (const float*)nullptr, (float2*)w.t1, (float2*)w.t2, (float2*)spec_out);
    if (rc) return rc;
    PB_CUDA_OK(cudaStreamSynchronize(ctx->stream));
    return POLYBIN_OK;
}

extern "C" int polybin_shell_maps(polybin_ctx* ctx, const void* spec, void* g_out) {
    if (!ctx || !spec || !g_out) return fail(ctx, POLYBIN_EINVAL, "polybin_shell_maps: NULL argument");
    int rc;
    Work& w = ctx->w;
    if (ctx->prec == POLYBIN_FP64) {
        if ((rc = ensure_fine_inv<double>(ctx))) return rc;
        rc = run_shells<double>(ctx, (const double2*)spec, (double2*)w.u1f, (double2*)w.u2f, (double*)g_out, 0, ctx->fg);
    } else {
        if ((rc = ensure_fine_inv<float>(ctx))) return rc;
        rc = run_shells<float>(ctx, (const float2*)spec, (float2*)w.u1f, (float2*)w.u2f, (float*)g_out, 0, ctx->fg);
    }
    if (rc) return rc;
    PB_CUDA_OK(cudaStreamSynchronize(ctx->stream));
    return POLYBIN_OK;
}

extern "C" int polybin_contract(polybin_ctx* ctx, const void* g, int n_g, const void* h, int n_h, double* m_out) {
    if (!ctx || !g || !m_out) return fail(ctx, POLYBIN_EINVAL, "polybin_contract: NULL argument");
    if (!h) n_h = n_g;
    if (n_g < 1 || n_g > 64 || n_h < 1 || n_h > 64) return fail(ctx, POLYBIN_EINVAL, "polybin_contract: 1 <= n_g, n_h <= 64");
    int rc;
    Work& w = ctx->w;
    const size_t nout = (size_t)n_g * (n_g + 1) / 2 * n_h;
    if (ctx->prec == POLYBIN_FP64)
        rc = run_contract_any<double>(ctx, (const double*)g, n_g, (const double*)h, n_h, w.partial, w.partial_cap, w.mout,
                                      ctx->ncell);
    else
        rc = run_contract_any<float>(ctx, (const float*)g, n_g, (const float*)h, n_h, w.partial, w.partial_cap, w.mout,
                                     ctx->ncell);
    if (rc) return rc;
    PB_CUDA_OK(cudaMemcpyAsync(m_out, w.mout, sizeof(double) * nout, cudaMemcpyDeviceToHost, ctx->stream));
    PB_CUDA_OK(cudaStreamSynchronize(ctx->stream));
    return POLYBIN_OK;
}

extern "C" int polybin_bk_pk_ideal(polybin_ctx* ctx, const float* delta, int batch, double* bk_out, double* pk_out) {
    if (!ctx || !delta || batch < 0) return fail(ctx, POLYBIN_EINVAL, "polybin_bk_pk_ideal: bad argument");
    int rc;
    if (bk_out && (rc = ensure_triplets(ctx))) return rc;
    return ctx->prec == POLYBIN_FP64 ? bk_pk_t<double>(ctx, delta, batch, bk_out, pk_out)
                                     : bk_pk_t<float>(ctx, delta, batch, bk_out, pk_out);
}

extern "C" int polybin_set_profiling(polybin_ctx* ctx, int on) {
    if (!ctx) return fail(ctx, POLYBIN_EINVAL, "polybin_set_profiling: NULL context");
    if (on && !ctx->tev[0]) {
        for (int i = 0; i < 2 * polybin_ctx::kTimerSlots; ++i) {
            cudaError_t e = cudaEventCreate(&ctx->tev[i]);
            if (e != cudaSuccess) {
                for (int j = 0; j < i; ++j) cudaEventDestroy(ctx->tev[j]);
                for (int j = 0; j < i; ++j) ctx->tev[j] = nullptr;
                return fail_cuda(ctx, e, "cudaEventCreate", __FILE__, __LINE__);
            }
        }
    }
    ctx->profiling = on != 0;
    return POLYBIN_OK;
}

extern "C" int polybin_get_stage_times(polybin_ctx* ctx, double* ms, long long* calls, int reset) {
    if (!ctx || !ms) return fail(ctx, POLYBIN_EINVAL, "polybin_get_stage_times: NULL argument");
    harvest_stage_times(ctx);
    for (int s = 0; s < kNumStages; ++s) {
        ms[s] = ctx->stage_ms[s];
        if (calls) calls[s] = ctx->stage_calls[s];
        if (reset) { ctx->stage_ms[s] = 0; ctx->stage_calls[s] = 0; }
    }
    return POLYBIN_OK;
}

extern "C" int polybin_launch_count(const polybin_ctx* ctx, long long* n) {
    if (!ctx || !n) return fail(const_cast<polybin_ctx*>(ctx), POLYBIN_EINVAL, "polybin_launch_count: NULL argument");
    *n = ctx->launches;
    return POLYBIN_OK;
}
