// Tensor-core (tcgen05, sm_103a) triplet contraction with 3-term split-TF32 products.
//
// Computes M[p][i] = sum_x P_p(x) h_i(x), P_p = g_j g_k for pairs p = (j <= k), as the GEMM
// D[128-row pair tile][32 singles] += A[pairs][cells] . B[singles][cells]^T over the cells of each CTA
// (Sec. 4.3.1, eq. beta-def: the real-space sum of the separable bispectrum; with h = g, S_abc for all
// a <= b and all c).  Each value v is split as v = hi + lo with hi = rna_tf32(v), lo = v - hi, and the
// product is accumulated as hi_a hi_b + hi_a lo_b + lo_a hi_b (the lo_a lo_b term, ~2^-22 relative, is
// dropped).
//
// Work split: a CTA takes one contiguous range of cells and one row group of two 128-row pair tiles (256
// pairs); two CTAs run on each SM (the grid covers 2 x 152 CTAs over row groups and cell ranges), so two
// independent producer/MMA pipelines overlap each other's handshake latency.
//
// Warp roles (256 threads per CTA):
//   warps 0-3   producers: stream the map tiles into a shared-memory ring with cp.async, form the pair
//               products (a thread owns one TMEM lane, i.e. one row of both pair tiles), split them and write
//               them into TMEM with tcgen05.st (the A operand never touches shared memory), and convert the
//               singles tile to hi/lo TF32 in the canonical no-swizzle K-major layout (the B operand).
//   warps 4-7   epilogue: every kPeriod chunks (64 cells) read the accumulators with tcgen05.ld into FP32
//               register sums (round-to-nearest), every kSpill periods add those into FP64 partials in
//               shared memory; finally write the CTA's FP64 partials.  Warp 4 allocates TMEM.  Lane 0 of
//               warps 4 and 5 issues the tcgen05.mma (A from TMEM, B from shared memory, D in TMEM) and the
//               tcgen05.commit of one pair tile for period q before its warp drains period q-1 (D is double
//               buffered); the 128x32x8 MMAs are short, so one issuing thread per tile keeps more in flight.
// Precision: the tensor core's internal accumulation is not round-to-nearest, so its error grows with the
// number of MMAs accumulated into one D; the 64-cell periods keep that chain at 24 MMAs.
// TMEM (256 columns per CTA): D double buffer 2 x (2 tiles x 32 columns) at [0, 128); A ring = 2 stages x
// (2 tiles x (16 hi + 16 lo)) at [128, 256).  Every mbarrier wait is bounded; on timeout the CTA raises an
// error flag and exits after draining its own asynchronous work.
#include <cuda_runtime.h>

#include <algorithm>

#include "polybin_internal.h"

namespace pb {
namespace tc {

constexpr int kKC = 16;           // cells per chunk (two K=8 MMA steps)
constexpr int kStages = 2;        // A/B pipeline depth
constexpr int kRing = 4;          // map-tile ring (prefetch distance 3)
constexpr int kPeriod = 4;        // chunks per tensor-memory accumulation period (64 cells)
constexpr int kSpill = 32;        // periods per FP32 register accumulation before the FP64 update (2048 cells)
constexpr int kMaxTiles = 4;      // pair tiles of 128 rows over all row groups (npairs <= 512)
constexpr int kTiles = 2;         // pair tiles per CTA (a row group of 256 pairs); two CTAs per SM
constexpr int kNCols = 32;        // singles per tile (nh <= 32)
constexpr int kGS = 20;           // floats per map row in the ring (16 + 4 pad: conflict-free LDS.128)
constexpr int kProducerWarps = 4;
constexpr int kProducers = 32 * kProducerWarps;
constexpr int kMmaWarp = kProducerWarps;   // first epilogue warp; allocates TMEM
constexpr int kIssuers = kTiles;           // epilogue warps 4, 5: lane 0 issues the MMAs of tile (warp - 4)
constexpr int kEpilogue = 128;             // 4 epilogue warps
constexpr int kThreads = kProducers + kEpilogue;
constexpr int kTmemCols = 256;             // D 2 x (2 tiles x 32) at [0, 128); A 2 stages x (2 tiles x 32) at [128, 256)
constexpr unsigned kSpinLimit = 1u << 22;

struct Params {
    const float* g;
    const float* h;        // may equal g
    long ncell;
    long cells_cta;
    int ng, nh, npairs, ntiles;
    const short2* pairs;
    double* partial;       // [gridDim.x][npairs][nh]
    int* err;              // set to 1 on a timed-out wait
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait; returns false (and raises the abort flag) if the phase did not complete in time or another
// role aborted.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag, int* err,
                                          int backoff) {
    for (unsigned it = 0; it < kSpinLimit; ++it) {
        if (mbar_try(bar, parity)) return true;
        if (*abort_flag) return false;
        if (backoff) __nanosleep(64);
    }
    *abort_flag = 1;
    atomicExch(err, 1);
    return false;
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ uint32_t to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

// v = hi + lo with hi = rna_tf32(v) and lo = v - hi exact in FP32; the MMA reads lo's leading 11 bits.
__device__ __forceinline__ void split2(float v, uint32_t& hi, uint32_t& lo) {
    hi = to_tf32(v);
    lo = __float_as_uint(v - __uint_as_float(hi));
}

__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t* v) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16};" ::"r"(taddr),
        "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]),
        "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15])
        : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t* v) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
          "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
          "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(taddr)
        : "memory");
}

// Shared-memory matrix descriptor, no swizzle (canonical K-major "interleaved" layout): core matrices of
// 8 rows x 16 bytes; LBO = byte distance between core matrices adjacent in K, SBO = between 8-row groups.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;   // descriptor version for tcgen05
    return d;                 // base offset 0, layout type 0 (no swizzle)
}

// Instruction descriptor: kind::tf32, D = F32, A = B = TF32, both K-major, M = 128, N = 32.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint32_t a_tmem, uint64_t b_desc, uint32_t idesc,
                                         uint32_t accum) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
        "r"(a_tmem), "l"(b_desc), "r"(idesc), "r"(accum)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// Named-barrier AND-vote over the 128 producer threads (barrier 1): every producer gets the same answer.
__device__ __forceinline__ bool producers_all(bool v) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\tbar.red.and.pred q, 1, 128, p;\n\tselp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)v)
        : "memory");
    return r != 0;
}

__device__ __forceinline__ void cp_async16(void* dst, const void* src, int src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(src_bytes)
                 : "memory");
}

__global__ void __launch_bounds__(kThreads, 2) k_contract_tc(Params P) {
    extern __shared__ __align__(1024) unsigned char smem[];
    double* acc64 = reinterpret_cast<double*>(smem);                                   // [kTiles][32][128]
    unsigned char* bbase = smem + (size_t)kTiles * kNCols * 128 * sizeof(double);      // B stages
    const int BSTAGE = 2 * kNCols * kKC * 4;                                            // hi + lo, 4 KB
    float* ring = reinterpret_cast<float*>(bbase + kStages * BSTAGE);                   // [kRing][rows][kGS]
    const int rows = P.ng + (P.h != P.g ? P.nh : 0);
    uint64_t* bars = reinterpret_cast<uint64_t*>(ring + (size_t)kRing * rows * kGS);
    uint64_t* full = bars;                  // [kStages]   producers -> MMA
    uint64_t* empty = bars + kStages;       // [kStages]   MMA commit -> producers
    uint64_t* dfull = bars + 2 * kStages;   // [2]         MMA commit -> epilogue
    uint64_t* dempty = dfull + 2;           // [2]         epilogue -> MMA
    uint64_t* fin = dempty + 2;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(fin + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const long cbeg = (long)blockIdx.x * P.cells_cta;
    const int rg = blockIdx.y;                                  // row group: pair tiles 2 rg, 2 rg + 1
    const int ntl = min(kTiles, P.ntiles - kTiles * rg);        // tiles of this CTA
    const long cend = min(P.ncell, cbeg + P.cells_cta);
    const int nchunks = cbeg < cend ? (int)((cend - cbeg + kKC - 1) / kKC) : 0;
    const int nperiods = (nchunks + kPeriod - 1) / kPeriod;

    for (int i = tid; i < kTiles * kNCols * 128; i += blockDim.x) acc64[i] = 0.0;
    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) { mbar_init(&full[s], kProducers); mbar_init(&empty[s], kIssuers); }
        for (int d = 0; d < 2; ++d) { mbar_init(&dfull[d], kIssuers); mbar_init(&dempty[d], kEpilogue); }
        mbar_init(fin, kIssuers);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == kMmaWarp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(smem_u32(tmem_slot)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;        // D buffer d, tile t at column 64 d + 32 t
    const uint32_t A0 = tmem + 128;          // A stage s, tile t: hi at 128 + 64 s + 32 t, lo at +16

    if (warp < kProducerWarps) {
        // ------------------------------------------------------------------ producers
        const bool hsep = P.h != P.g;
        const int quarter = warp & 3;
        const int row = 32 * quarter + lane;
        const uint32_t lane_base = (uint32_t)(32 * quarter) << 16;
        int pj[kTiles], pk[kTiles];
#pragma unroll
        for (int u = 0; u < kTiles; ++u) {
            const int p = 128 * (kTiles * rg + u) + row;
            if (u < ntl && p < P.npairs) { short2 jk = P.pairs[p]; pj[u] = jk.x; pk[u] = jk.y; }
            else { pj[u] = -1; pk[u] = -1; }
        }
        auto issue = [&](int c) {
            if (c < nchunks) {
                float* slot = ring + (size_t)(c % kRing) * rows * kGS;
                const long x0 = cbeg + (long)c * kKC;
                for (int q = tid; q < rows * 4; q += kProducers) {
                    const int r = q >> 2, quad = q & 3;
                    const float* src = (r < P.ng) ? P.g + (long)r * P.ncell : P.h + (long)(r - P.ng) * P.ncell;
                    const long cell = x0 + quad * 4;
                    const long valid = min(4L, max(0L, cend - cell));
                    cp_async16(slot + r * kGS + quad * 4, valid > 0 ? src + cell : src, (int)(valid * 4));
                }
            }
            asm volatile("cp.async.commit_group;" ::: "memory");
        };
        issue(0);
        issue(1);
        issue(2);
        bool ok = true;
        for (int c = 0; c < nchunks; ++c) {
            const int s = c % kStages;
            asm volatile("cp.async.wait_group 2;" ::: "memory");
            bool mine = true;
            if (c >= kStages) mine = mbar_wait(&empty[s], (uint32_t)((c / kStages - 1) & 1), abort_flag, P.err, 0);
            // uniform decision + barrier: chunk c's tile is visible to all producers and chunk c-1 is finished
            ok = producers_all(mine);
            if (!ok) break;
            if (c >= kStages) tc_fence_after();
            issue(c + 3);
            const float* tile = ring + (size_t)(c % kRing) * rows * kGS;
            // A operand: pair products split into TF32 hi and FP32 remainder (read as TF32 by the MMA), into TMEM
#pragma unroll
            for (int u = 0; u < kTiles; ++u) {
                const int t = u;
                if (t >= ntl) break;
                uint32_t hi[kKC], lo[kKC];
                if (pj[u] >= 0) {
                    const float4* a = reinterpret_cast<const float4*>(tile + pj[u] * kGS);
                    const float4* b = reinterpret_cast<const float4*>(tile + pk[u] * kGS);
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const float4 x = a[q], y = b[q];
                        split2(x.x * y.x, hi[4 * q + 0], lo[4 * q + 0]);
                        split2(x.y * y.y, hi[4 * q + 1], lo[4 * q + 1]);
                        split2(x.z * y.z, hi[4 * q + 2], lo[4 * q + 2]);
                        split2(x.w * y.w, hi[4 * q + 3], lo[4 * q + 3]);
                    }
                } else {
#pragma unroll
                    for (int q = 0; q < kKC; ++q) { hi[q] = 0u; lo[q] = 0u; }
                }
                const uint32_t col = 128u + 64u * s + 32u * t;
                tmem_st16(tmem + lane_base + col, hi);
                tmem_st16(tmem + lane_base + col + 16u, lo);
            }
            // B operand (threads 0..127): singles hi/lo in the no-swizzle K-major layout:
            // element (row r, cell k) at (r / 8) * 512 + (k / 4) * 128 + (r % 8) * 16 + (k % 4) * 4 bytes.
            if (tid < 128) {
                unsigned char* bs = bbase + s * BSTAGE;
                const int r = tid >> 2, quad = tid & 3;
                uint4 vh = make_uint4(0, 0, 0, 0), vl = make_uint4(0, 0, 0, 0);
                if (r < P.nh) {
                    const int rr = hsep ? P.ng + r : r;
                    const float4 v = *reinterpret_cast<const float4*>(tile + rr * kGS + quad * 4);
                    split2(v.x, vh.x, vl.x);
                    split2(v.y, vh.y, vl.y);
                    split2(v.z, vh.z, vl.z);
                    split2(v.w, vh.w, vl.w);
                }
                const int off = (r >> 3) * 512 + quad * 128 + (r & 7) * 16;
                *reinterpret_cast<uint4*>(bs + off) = vh;
                *reinterpret_cast<uint4*>(bs + 2048 + off) = vl;
            }
            asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            tc_fence_before();
            mbar_arrive(&full[s]);
        }
        asm volatile("cp.async.wait_all;" ::: "memory");
        if (!ok) *abort_flag = 1;
    } else {
        // ------------------------------------------------------------------ epilogue (+ MMA issue in warp 8)
        const int quarter = warp & 3;              // TMEM lane quarter this warp may access
        const int row = 32 * quarter + lane;
        const uint32_t lane_base = (uint32_t)(32 * quarter) << 16;
        const int iidx = warp - kMmaWarp;
        const bool issuer = iidx < kIssuers;
        float acc[kTiles][kNCols];
#pragma unroll
        for (int u = 0; u < kTiles; ++u)
#pragma unroll
            for (int i = 0; i < kNCols; ++i) acc[u][i] = 0.f;
        auto spill = [&]() {
#pragma unroll
            for (int u = 0; u < kTiles; ++u) {
                const int t = u;
                if (t >= ntl) break;
#pragma unroll
                for (int i = 0; i < kNCols; ++i) {
                    acc64[(t * kNCols + i) * 128 + row] += (double)acc[u][i];
                    acc[u][i] = 0.f;
                }
            }
        };
        // read the accumulators of period q, release the D buffer, add into the FP32 register sums
        auto drain = [&](int q) -> bool {
            const int d = q & 1;
            if (!mbar_wait(&dfull[d], (uint32_t)((q >> 1) & 1), abort_flag, P.err, issuer ? 0 : 1)) return false;
            tc_fence_after();
#pragma unroll
            for (int u = 0; u < kTiles; ++u) {
                const int t = u;
                if (t >= ntl) break;
                uint32_t v[kNCols];
                tmem_ld32(tmem + lane_base + 64u * d + 32u * t, v);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int i = 0; i < kNCols; ++i) acc[u][i] += __uint_as_float(v[i]);
            }
            tc_fence_before();
            mbar_arrive(&dempty[d]);
            if ((q + 1) % kSpill == 0) spill();
            return true;
        };
        // issue the MMAs of period q (lane 0 of the issuer warp)
        bool mma_ok = true;
        auto issue_period = [&](int q) {
            const uint32_t idesc = idesc_tf32(128, kNCols);
            const uint32_t bstage0 = smem_u32(bbase);
            const int d = q & 1;
            if (q >= 2 && !mbar_wait(&dempty[d], (uint32_t)((q / 2 - 1) & 1), abort_flag, P.err, 0)) { mma_ok = false; return; }
            const int c1 = min(nchunks, (q + 1) * kPeriod);
            for (int c = q * kPeriod; c < c1; ++c) {
                const int s = c % kStages;
                const bool first = c == q * kPeriod;
                if (!mbar_wait(&full[s], (uint32_t)((c / kStages) & 1), abort_flag, P.err, 0)) { mma_ok = false; return; }
                tc_fence_after();
                const uint32_t bh = bstage0 + s * BSTAGE, bl = bh + 2048;
                for (int t = iidx; t < ntl; t += kIssuers) {
                    const uint32_t dcol = tmem + 64u * d + 32u * t;
                    const uint32_t ah = A0 + 64u * s + 32u * t, al = ah + 16u;
#pragma unroll
                    for (int ks = 0; ks < kKC / 8; ++ks) {
                        const uint64_t dbh = sdesc(bh + ks * 256, 128, 512);
                        const uint64_t dbl = sdesc(bl + ks * 256, 128, 512);
                        mma_tf32(dcol, ah + 8u * ks, dbh, idesc, (first && ks == 0) ? 0u : 1u);
                        mma_tf32(dcol, ah + 8u * ks, dbl, idesc, 1u);
                        mma_tf32(dcol, al + 8u * ks, dbh, idesc, 1u);
                    }
                }
                mma_commit(&empty[s]);
            }
            mma_commit(&dfull[d]);
        };
        bool ok = true;
        if (issuer) {
            for (int q = 0; q < nperiods; ++q) {
                if (lane == 0 && mma_ok) issue_period(q);
                __syncwarp();
                if (q >= 1 && ok) ok = drain(q - 1);
            }
            if (nperiods >= 1 && ok) ok = drain(nperiods - 1);
            if (lane == 0) {
                // every MMA issued by this thread has completed before TMEM is released
                mma_commit(fin);
                for (unsigned it = 0; it < kSpinLimit && !mbar_try(fin, 0); ++it) {
                }
                if (!mma_ok) *abort_flag = 1;
            }
            __syncwarp();
        } else {
            for (int q = 0; q < nperiods && ok; ++q) ok = drain(q);
        }
        spill();
        for (int u = 0; u < kTiles; ++u) {
            const int t = u;
            if (t >= ntl) break;
            const int p = 128 * (kTiles * rg + t) + row;
            if (p >= P.npairs) continue;
            double* out = P.partial + ((size_t)blockIdx.x * P.npairs + p) * P.nh;
            for (int i = 0; i < P.nh; ++i) out[i] = acc64[(t * kNCols + i) * 128 + row];
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == kMmaWarp) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tmem));
}

// Self-test of the bounded waits: one thread waits on an mbarrier phase that nothing completes; the wait gives up
// after `limit` polls and raises the error flag, as a stalled pipeline would, and the kernel returns normally.
__global__ void k_wait_selftest(int* err, unsigned limit) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        unsigned it = 0;
        for (; it < limit; ++it)
            if (mbar_try(&bar, 0)) break;
        if (it == limit) atomicExch(err, 1);
    }
}

}  // namespace tc

bool split_tc_available() { return true; }

int ensure_err_flag(polybin_ctx* ctx) {
    if (ctx->d_err) return POLYBIN_OK;
    cudaError_t e = cudaMalloc(&ctx->d_err, sizeof(int));
    if (e != cudaSuccess) return fail_cuda(ctx, e, "cudaMalloc err flag", __FILE__, __LINE__);
    e = cudaMemset(ctx->d_err, 0, sizeof(int));
    if (e != cudaSuccess) return fail_cuda(ctx, e, "cudaMemset err flag", __FILE__, __LINE__);
    return POLYBIN_OK;
}

static size_t tc_smem_bytes(int rows) {
    return (size_t)tc::kTiles * tc::kNCols * 128 * sizeof(double) + tc::kStages * 2 * tc::kNCols * tc::kKC * 4 +
           (size_t)tc::kRing * rows * tc::kGS * sizeof(float) + 256;
}

// Geometry of the tensor-core contraction: one CTA per SM over a contiguous cell range.
ContractGeom contract_geom_tc(int ng, int nh, long ncell) {
    ContractGeom G;
    G.nb = ng; G.nh = nh; G.npairs = ng * (ng + 1) / 2;
    G.rt = G.ct = 0; G.rows_cta = 128; G.nhp = tc::kNCols;
    G.ngroups = (G.npairs + 127) / 128;                 // pair tiles; a CTA takes kTiles of them
    const int nrg = (G.ngroups + tc::kTiles - 1) / tc::kTiles;
    const long nchunk = (ncell + tc::kKC - 1) / tc::kKC;
    const long ncta = std::max(1L, std::min(304L / nrg, nchunk));   // two CTAs per SM over all row groups
    G.cells_cta = ((ncell + ncta - 1) / ncta + tc::kKC - 1) / tc::kKC * tc::kKC;
    G.ncb = (int)((ncell + G.cells_cta - 1) / G.cells_cta);
    return G;
}

int run_contract_tc(polybin_ctx* ctx, const float* g, int ng, const float* h, int nh, double* d_partial,
                    size_t partial_cap, double* d_out) {
    if (!h) { h = g; nh = ng; }
    ContractGeom G = contract_geom_tc(ng, nh, ctx->ncell);
    if ((size_t)G.ncb * G.npairs * G.nh > partial_cap) return fail(ctx, POLYBIN_EINVAL, "contract_tc: partial buffer too small");
    if (ctx->ncell % 4) return fail(ctx, POLYBIN_EINVAL, "contract_tc: the number of cells must be a multiple of 4");
    int rc0 = ensure_err_flag(ctx);
    if (rc0) return rc0;
    cudaError_t e = cudaMemsetAsync(ctx->d_err, 0, sizeof(int), ctx->stream);
    if (e != cudaSuccess) return fail_cuda(ctx, e, "cudaMemsetAsync", __FILE__, __LINE__);
    const int rows = ng + (h != g ? nh : 0);
    const size_t sm = tc_smem_bytes(rows);
    e = cudaFuncSetAttribute((const void*)tc::k_contract_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return fail_cuda(ctx, e, "cudaFuncSetAttribute(k_contract_tc)", __FILE__, __LINE__);
    tc::Params P;
    P.g = g; P.h = h; P.ncell = ctx->ncell; P.cells_cta = G.cells_cta;
    P.ng = ng; P.nh = nh; P.npairs = G.npairs; P.ntiles = G.ngroups;
    P.pairs = ctx->d_pairs + pairs_offset(ng);
    P.partial = d_partial;
    P.err = ctx->d_err;
    {
        StageTimer timer(ctx, kStageContract);
        const int nrg = (G.ngroups + tc::kTiles - 1) / tc::kTiles;
        tc::k_contract_tc<<<dim3(G.ncb, nrg, 1), tc::kThreads, sm, ctx->stream>>>(P);
        ctx->launches += 1;
        e = cudaGetLastError();
        if (e != cudaSuccess) return fail_cuda(ctx, e, "k_contract_tc", __FILE__, __LINE__);
        const long nout = (long)G.npairs * G.nh;
        k_reduce_partials<<<(unsigned)((nout + 255) / 256), 256, 0, ctx->stream>>>(d_partial, G.ncb, nout, d_out);
        ctx->launches += 1;
        e = cudaGetLastError();
        if (e != cudaSuccess) return fail_cuda(ctx, e, "k_reduce_partials", __FILE__, __LINE__);
    }
    if (ctx->capturing) return POLYBIN_OK;   // the caller reads the error flag after the graph has run
    int herr = 0;
    e = cudaMemcpyAsync(&herr, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return fail_cuda(ctx, e, "contract_tc error flag", __FILE__, __LINE__);
    if (herr) return fail(ctx, POLYBIN_ETIMEOUT, "contract_tc: a pipeline wait timed out");
    return POLYBIN_OK;
}

}  // namespace pb

extern "C" int polybin_selftest_wait(polybin_ctx* ctx, int* timed_out) {
    if (!ctx || !timed_out) return pb::fail(ctx, POLYBIN_EINVAL, "polybin_selftest_wait: NULL argument");
    int rc = pb::ensure_err_flag(ctx);
    if (rc) return rc;
    PB_CUDA_OK(cudaMemsetAsync(ctx->d_err, 0, sizeof(int), ctx->stream));
    pb::tc::k_wait_selftest<<<1, 32, 0, ctx->stream>>>(ctx->d_err, 1u << 14);
    ctx->launches++;
    PB_CUDA_OK(cudaGetLastError());
    PB_CUDA_OK(cudaMemcpyAsync(timed_out, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    PB_CUDA_OK(cudaStreamSynchronize(ctx->stream));
    return POLYBIN_OK;
}
