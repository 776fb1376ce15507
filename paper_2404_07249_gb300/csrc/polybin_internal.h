// Internal declarations shared by the translation units of libpolybin (not part of the C-ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "common.cuh"
#include "contract.cuh"
#include "fft.cuh"
#include "polybin.h"

#define PB_CUDA_OK_C(expr) PB_CUDA_OK(expr)

namespace pb {

// Per-bin bounding box of the inverse transforms and offsets of its intermediates.
struct BinBox {
    AxisRange rx, ry, rz;
    long u1_off, u2_off;
};

// A grid the shell maps are evaluated on: its lengths, FFT plans and twiddles, and every bin's bounding box with
// the offsets of that bin's inverse-transform intermediates.  Two are kept per context: the data grid (maps
// returned to the caller, maps that are multiplied by a mask in real space) and the contraction grid, the
// smallest 2-3-5 grid on which the triple product of three band-limited maps is alias-free (see plan_bins).
struct InvGrid {
    int N[3] = {0, 0, 0};
    long ncell = 0;
    FftPlan plan[3];
    const void* tw_f[3] = {nullptr, nullptr, nullptr};   // float2 e^{-2 pi i m / N_a}
    const void* tw_d[3] = {nullptr, nullptr, nullptr};   // double2
    std::vector<BinBox> bbox;
    long u1_total = 0, u2_total = 0;
};

// Device workspace of one compute precision.
struct Work {
    size_t elem = 0;
    void* t1 = nullptr;      // forward z-pass output [N0*N1][Bz]
    void* t2 = nullptr;      // forward y-pass output [N0][By][Bz]
    void* box = nullptr;     // pruned spectrum [Bx][By][Bz]
    void* u1 = nullptr;      // inverse x-pass outputs, all bins (contraction grid)
    void* u2 = nullptr;      // inverse y-pass outputs, all bins (contraction grid)
    void* u1f = nullptr;     // the same on the data grid, allocated on first use (ensure_fine_inv)
    void* u2f = nullptr;
    void* g = nullptr;       // shell maps [nb][cg.ncell] on the contraction grid
    void* g2 = nullptr;      // Legendre-weighted shell maps [nb][cg.ncell] (bispectrum multipoles), on first use
    double* partial = nullptr;
    size_t partial_cap = 0;
    double* mout = nullptr;  // contraction result [npairs][nh]
};

int fail(polybin_ctx* ctx, int status, const char* fmt, ...);
int fail_cuda(polybin_ctx* ctx, cudaError_t e, const char* what, const char* file, int line);

inline int pair_index(int nb, int a, int b) { return a * nb - a * (a - 1) / 2 + (b - a); }
__host__ __device__ inline long pairs_offset(int n) { return (long)(n - 1) * n * (n + 1) / 6; }  // sum_{m<n} m(m+1)/2

// Gaussian elimination with partial pivoting on an n x (n+1) augmented matrix (n <= 3).
inline bool solve_small(double A[3][4], int n, double* x) {
    for (int c = 0; c < n; ++c) {
        int p = c;
        for (int r = c + 1; r < n; ++r)
            if ((A[r][c] < 0 ? -A[r][c] : A[r][c]) > (A[p][c] < 0 ? -A[p][c] : A[p][c])) p = r;
        if (A[p][c] == 0.0) return false;
        if (p != c)
            for (int k = 0; k <= n; ++k) { double t = A[c][k]; A[c][k] = A[p][k]; A[p][k] = t; }
        for (int r = c + 1; r < n; ++r) {
            const double f = A[r][c] / A[c][c];
            for (int k = c; k <= n; ++k) A[r][k] -= f * A[c][k];
        }
    }
    for (int r = n - 1; r >= 0; --r) {
        double s = A[r][n];
        for (int k = r + 1; k < n; ++k) s -= A[r][k] * x[k];
        x[r] = s / A[r][r];
    }
    return true;
}

ContractGeom contract_geom(int nb, int nh, long ncell);

template <typename T, typename TIN, typename TM>
int run_forward(polybin_ctx*, const TIN*, const TM*, const TM*, C<T>*, C<T>*, C<T>*);
// The same on grid ig (the data grid ctx->fg or the contraction grid ctx->cg; intermediates sized for it).
template <typename T, typename TIN, typename TM>
int run_forward(polybin_ctx*, const TIN*, const TM*, const TM*, C<T>*, C<T>*, C<T>*, const InvGrid& ig);
// Shell maps of all bins on grid `ig` (the data grid ctx->fg or the contraction grid ctx->cg), normalised with the
// 1/N of the data grid's inverse DFT, so that maps on either grid sample the same band-limited function.
template <typename T> int run_shells(polybin_ctx*, const C<T>*, C<T>*, C<T>*, T*, int ell, const InvGrid& ig);
// The same with the weight Ybar_lm(k / |k|) of the local line of sight (m in [-ell, ell]; m = kLegendreM: L_ell(mu)).
template <typename T>
int run_shells_m(polybin_ctx*, const C<T>*, C<T>*, C<T>*, T*, int ell, int m, const InvGrid& ig);
template <typename T> int run_pkbin(polybin_ctx*, const C<T>*, std::vector<double>&);
// Contractions over `ncell` cells (maps of the data grid or of the contraction grid).
template <typename T> int run_contract(polybin_ctx*, const T*, int, const T*, int, double*, size_t, double*, long ncell);
// Contraction dispatch: the tensor-core kernel in POLYBIN_SPLIT_TF32X3 mode, the SIMT kernel otherwise.
template <typename T> int run_contract_any(polybin_ctx*, const T*, int, const T*, int, double*, size_t, double*, long ncell);
template <typename T> int alloc_work(polybin_ctx*, Work&);
// Data-grid intermediates of the inverse transforms (ctx->w.u1f, u2f), allocated on first use.
template <typename T> int ensure_fine_inv(polybin_ctx*);
int alloc_work_shells_double(polybin_ctx*, Work&);
void free_work(Work&);
int resolve_input(polybin_ctx*, const float*, size_t, const float**);
int ensure_triplets(polybin_ctx*);
bool split_tc_available();
int tf32_selfcheck(polybin_ctx*);
bool tc_shape_ok(long ncell, const float* g, int ng, const float* h, int nh);
int run_contract_tc(polybin_ctx*, const float*, int, const float*, int, double*, long ncell);
int prepare_triplet_tc(polybin_ctx*);
int run_triplet_sums_tc(polybin_ctx*, const float* g, double* d_S);
int run_triplet_sums_ell_tc(polybin_ctx*, const float* g, const float* gl, double* d_S);
int run_gram_tc(polybin_ctx*, const float* A, int nA, const float* B, int nB, long K, double scale, double* d_out);
void destroy_tc(polybin_ctx*);
// S'_abc of every closed triplet (device, triplet order) from the nb shell maps g on the contraction grid; the
// data-grid sum is S_abc = cg_ratio S'_abc.
template <typename T> int run_triplet_sums(polybin_ctx*, const T* g, double* d_S);
// S^ell'_abc = sum_x g_a g_b g_{c,ell} (gl: the maps g_{c,ell} = IFT[Theta_c L_ell D]) on the contraction grid.
template <typename T> int run_triplet_sums_ell(polybin_ctx*, const T* g, const T* gl, double* d_S);
// B_abc = fac scale S'_abc / T_abc on the device (FP64), scale = (V^2 / N^3) cg_ratio (fac = 2 ell + 1 for a
// multipole).
int run_bk_normalise(polybin_ctx*, const double* d_S, double* d_B, double fac = 1.0);
// P_ell(b) from the P binning partials on the device (FP64): (2 ell + 1) (V / N^2) num / N_b.
int run_pk_normalise(polybin_ctx*, double* d_P);
// Inverse transform of a box spectrum (the box of wave numbers |n_i| <= m) to a real map on the data grid with the
// 1/N of the inverse DFT and an optional pointwise multiplier on output; v1 [N0][By][Bz], v2 [N0][N1][Bz].
template <typename T> int run_inverse_box(polybin_ctx*, const C<T>* box, C<T>* v1, C<T>* v2, T* out, const T* mulout);
// Optimal weighting (optimal.cu): out = post (/ n_w) G[Phi pre v (/ n_w)] by preconditioned conjugate gradients, with
// G the inverse of Phi (IFT[P FT[.]] + n2_w / n_w^2) Phi on the cells with n_w > 0.  pre = null, pre_div = 1 gives
// S^-1 v; post_div = 1 gives S^-T v; pre = n gives S^-1 P v; post = n with post_div = 1 gives P^T S^-T v.
template <typename T, typename TIN, typename TOUT>
int opt_apply(polybin_ctx*, const TIN* v, const float* pre, int pre_div, const float* post, int post_div, TOUT* out);
// Identity of the configured optimal weighting (0 if none) and the statistics of the last solve.
uint64_t opt_hash(const polybin_ctx*);
void opt_stats(const polybin_ctx*, int* iters, double* relres);
void destroy_optimal(polybin_ctx*);
void destroy_extras(polybin_ctx*);
void destroy_unwindowed(polybin_ctx*);
void destroy_multi(polybin_ctx*);
// Device error flags of a context: [kErrPipeline] the tensor-core kernels' bounded waits (cleared before each of
// their launches), [kErrStaging] the bulk staging copies of the transform passes (cleared when reported).
constexpr int kErrPipeline = 0, kErrStaging = 1, kErrFlags = 2;
int ensure_err_flag(polybin_ctx*);
int read_err_flags(polybin_ctx*, const char* what);
int run_bulk_wait_selftest(polybin_ctx*, unsigned limit);

}  // namespace pb

struct polybin_ctx {
    int N[3] = {0, 0, 0};
    long ncell = 0;
    double L = 0, vol = 0, kf = 0;
    int nb = 0;
    std::vector<double> edges;
    int lmax = 0, nell = 1;
    int prec = 0;
    cudaStream_t stream = nullptr;
    std::string err;

    // planner
    pb::AxisRange gx{0, 0}, gy{0, 0}, gz{0, 0};
    pb::InvGrid fg;              // inverse transforms on the data grid
    pb::InvGrid cg;              // inverse transforms on the contraction grid
    double cg_ratio = 1.0;       // ncell / cg.ncell
    void* d_ctw[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};   // contraction-grid twiddles (f, d)
    int smax = 0;
    std::vector<int16_t> lut;
    std::vector<int> bin_slo, bin_shi;   // range of integer |n|^2 of each bin (bins are contiguous in |n|)
    int16_t* d_lut = nullptr;
    pb::FftPlan plan[3];
    void* d_tw_f[3] = {nullptr, nullptr, nullptr};
    void* d_tw_d[3] = {nullptr, nullptr, nullptr};
    short2* d_pairs = nullptr;   // pair tables for every n <= 64, table n at pairs_offset(n)

    // workspace
    pb::Work w;
    float* d_in = nullptr;
    size_t in_cap = 0;
    // batched host input: two device buffers filled on a copy stream, the copy of field f + 1 overlapping the
    // transforms of field f
    float* d_stage[2] = {nullptr, nullptr};
    size_t stage_cap = 0;
    cudaStream_t cstream = nullptr;
    cudaEvent_t ev_copied[2] = {nullptr, nullptr}, ev_used[2] = {nullptr, nullptr};

    // P_ell binning
    long nmodes = 0;
    int* d_offs = nullptr;
    double* d_coef = nullptr;
    int* d_bin_start = nullptr;
    double* d_pkpart = nullptr;
    double* d_pkout = nullptr;   // normalised P_ell [nell][nb]
    double* d_counts = nullptr;  // N_b
    int pk_seg_len = 0, pk_nseg = 0;
    std::vector<double> counts;
    std::vector<double> fish_disc;   // [nb][nell][nell]

    // closed triplets (lexicographic), T_abc and N_abc; on the device: S_abc and B_abc of the last field, T_abc
    bool trip_ready = false;
    std::vector<int> trip;
    std::vector<double> Tabc, Nabc;
    double* d_S = nullptr;
    double* d_B = nullptr;       // normalised bispectrum of the last field
    double* d_T = nullptr;       // T_abc (data grid)
    // tensor-core contraction plans; closed-triplet SIMT plans (FP32 / FP64 modes)
    void* tc = nullptr;
    void* simt = nullptr;

    // instrumentation: kernel launches issued, and (when enabled) per-stage device time from CUDA events.
    // Stage brackets are recorded without blocking into tev (start, stop pairs) and read back lazily: when the
    // slots run out, or when the caller asks for the times.
    long launches = 0;
    bool profiling = false;
    double stage_ms[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    long stage_calls[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    static constexpr int kTimerSlots = 64;
    cudaEvent_t tev[2 * kTimerSlots] = {};
    int tstage[kTimerSlots] = {};
    int tused = 0;        // slots recorded since the last read-back
    bool topen = false;   // a stage bracket is open (brackets do not nest)

    // observer of the local line of sight, box coordinates centred on the origin (Mpc/h)
    double observer[3] = {0.0, 0.0, 0.0};
    // the contraction kernel that ran last (polybin_contract_path values), -1 before the first contraction
    int last_path = -1;
    // device error flags of the kernels with bounded waits ([kErrFlags] ints)
    int* d_err = nullptr;
    // stream capture in progress: kernels are enqueued without host synchronisation or read-backs
    bool capturing = false;
    // unique id (contexts at a reused address get a new id) and the cached multi-field graph
    unsigned long long uid = 0;
    void* multi = nullptr;

    // extension slots (unwindowed estimators; optimal weighting)
    void* ext = nullptr;
    void* opt = nullptr;
};

namespace pb {
enum Stage { kStageForward = 0, kStageShells = 1, kStageContract = 2, kStagePk = 3, kNumStages = 4 };
// Adds the elapsed times of the recorded stage brackets to stage_ms / stage_calls (waits for their stop events).
inline void harvest_stage_times(polybin_ctx* ctx) {
    for (int i = 0; i < ctx->tused; ++i) {
        float ms = 0.f;
        if (cudaEventSynchronize(ctx->tev[2 * i + 1]) == cudaSuccess &&
            cudaEventElapsedTime(&ms, ctx->tev[2 * i], ctx->tev[2 * i + 1]) == cudaSuccess) {
            ctx->stage_ms[ctx->tstage[i]] += ms;
            ctx->stage_calls[ctx->tstage[i]] += 1;
        }
    }
    ctx->tused = 0;
}

// Brackets a pipeline stage with CUDA events on the context stream when profiling is enabled.  Recording does not
// block the host; stream captures are not bracketed.
struct StageTimer {
    polybin_ctx* ctx;
    int slot = -1;
    StageTimer(polybin_ctx* c, int s) : ctx(c) {
        if (!ctx->profiling || ctx->capturing || ctx->topen || !ctx->tev[0]) return;
        if (ctx->tused == polybin_ctx::kTimerSlots) harvest_stage_times(ctx);
        slot = ctx->tused++;
        ctx->tstage[slot] = s;
        ctx->topen = true;
        cudaEventRecord(ctx->tev[2 * slot], ctx->stream);
    }
    ~StageTimer() {
        if (slot < 0) return;
        cudaEventRecord(ctx->tev[2 * slot + 1], ctx->stream);
        ctx->topen = false;
    }
};
}  // namespace pb
