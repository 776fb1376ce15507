// Tensor-core (tcgen05, sm_103a) triplet contraction with 3-term split-TF32 products.
//
// Computes sums M[(j, k)][i] = sum_x g_j(x) g_k(x) h_i(x) over the cells x (Sec. 4.3.1, eq. beta-def: the
// real-space sum of the separable bispectrum; with h = g the entry of pair (b, c) and single a is S_abc).  The work
// is a set of 128-row tiles: every row is one pair (j, k) and every tile has a window of W singles
// [s0, s0 + W), W in {16, 32}.  For the ideal bispectrum only the pairs and singles of closed triplets enter:
// the triplet a <= b <= c is read from pair (b, c) and single a, which prunes the 465 pairs x 30 singles of a
// 30-bin binning to 255 pairs in two tiles with windows of 16 and 32 singles.
//
// Arithmetic: A = pair products g_j g_k (FP32), split as A = A_hi + A_lo with A_hi = A rounded to TF32 (nearest,
// ties away from zero) and A_lo = A - A_hi in FP32 (read by the MMA as TF32).  B = singles: the tensor core reads an
// FP32 operand as TF32 by truncation (measured: the 13 low bits are dropped toward zero), so the raw maps in the TMA
// ring serve as B_hi = trunc(g) directly, and B_lo = g - trunc(g), rounded to TF32, is made per stage.  Per tile
// and K = 8 cells three MMAs of N = W run:  D[:, 0:W] += A_hi . B_hi^T  and  D[:, W:2W] += A_hi . B_lo^T +
// A_lo . B_hi^T  (both corrections in one accumulator); the lo*lo term (~2^-21 relative, unbiased) is dropped.  The
// tensor core's internal accumulation is not round-to-nearest, so D restarts every 64 cells (8 MMAs per hi*hi
// column); the epilogue adds D into FP32 registers (round-to-nearest) and those into FP64 shared memory every 2048
// cells.  Cross-CTA sums are FP64 in a fixed order (deterministic).
//
// Measured on this part (and shaping the design): an MMA issued from warp-uniform code with its operands in uniform
// registers costs ~16-20 cycles at N = 32 (the tensor pipe's rate), but ~200 cycles from a one-lane branch, so the
// issuing loops are warp-uniform (elect.sync inside the asm) and divide-free; MMAs into one accumulator back to back
// run at full rate; tensor memory stores reach ~650 B/clk an SM; the producers' shared-memory gathers (~500
// wavefronts a stage) and their latency set the stage time.  Tensor memory (512 columns) holds the accumulator
// (2W columns a tile) and a ring of A stages (64 columns a tile a stage).
//
// One CTA per SM over a contiguous range of cells, in stages of 32 cells (one TMA ring slot).  Warp roles, by
// warpgroup (setmaxnreg moves registers from warpgroup 0 to the producers):
//   warp 0       TMEM allocation; lane 0 streams the maps with TMA (cp.async.bulk.tensor, 32 cells x all maps per
//                load, 128-byte swizzle) into an 8-slot shared-memory ring.
//   warps 1-3    MMA issue: warp 1 + t waits for the stage (converged) and issues tile t's MMAs, commits them to the
//                stage's release barriers (A stage, ring slot) and, at a period's end, to the accumulator barrier.
//   warps 4-11   producers, two groups of four warps; group g makes cells 16g..16g+15 of every stage.  A thread owns
//                one TMEM lane, i.e. one row of every tile: it forms the pair products, splits them (packed FP32
//                pairs) and writes hi / lo straight into tensor memory (tcgen05.st: the A operand never touches
//                shared memory), loading the next tile's operands before forming the current tile's products; each
//                thread also makes one 16-byte chunk of the stage's B_lo.
//   warps 12-15  epilogue: after every period read D with tcgen05.ld (each warp its TMEM lane quarter), release
//                it to the issuers, accumulate.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <cstdlib>
#include <map>
#include <mutex>
#include <set>
#include <tuple>
#include <vector>

#include "polybin_internal.h"

namespace pb {
namespace tc {

constexpr int kSlotCells = 32;     // cells per TMA box row (128 bytes)
constexpr int kRingSlots = 8;
constexpr int kKC = 32;            // cells per A stage = one ring slot (four K = 8 MMA steps)
constexpr int kMaxAStages = 6;
constexpr int kPeriod = 2;         // A stages per TMEM accumulation period (64 cells)
constexpr int kSpill = 32;         // periods per FP32 register sum (2048 cells)
constexpr int kDBuf = 1;           // accumulator buffers (1: the issuers wait for the epilogue between periods)
static_assert(kDBuf == 1, "the MMA issue loop assumes one accumulator buffer");
constexpr int kMaxTiles = 3;       // tiles per CTA
constexpr int kMaxUnits = 3;       // 16-column output units per CTA (16 FP32 sums each, in registers)
constexpr int kMaxGroups = 4;      // row groups (grid.y)
constexpr int kProdGroups = 2;     // producer warp groups; group g makes half g (16 cells) of every stage
constexpr int kProdWarps = 4 * kProdGroups;
constexpr int kEpiWarps = 4;
// Warpgroup 0: TMA (warp 0), MMA issue (warp 1), two idle warps; warpgroups 1-2: producers; warpgroup 3: epilogue.
constexpr int kProdWarp0 = 4;
constexpr int kWarps = 16;
// Register split (setmaxnreg, per warpgroup): the CTA is launched with 128 registers a thread (65536 in all);
// warpgroup 0 gives registers back, the producers take them, the epilogue keeps 128:
// 48 * 128 + 168 * 256 + 128 * 128 = 65536.
constexpr int kRegsLaunch = 128, kRegsCtl = 48, kRegsProd = 168;
static_assert(kRegsCtl * 128 + kRegsProd * 256 + kRegsLaunch * 128 <= kRegsLaunch * 32 * kWarps,
              "register split exceeds the launch allocation");
constexpr int kThreads = 32 * kWarps;
constexpr int kMinSmem = 120 * 1024;   // one CTA per SM (the CTA allocates all 512 TMEM columns)
constexpr unsigned kSpinLimit = 1u << 22;
constexpr int kBloItems = 2;       // B_lo chunks per producer thread: <= 64 singles rows x 8 chunks / 256 threads

struct GroupDesc {
    int tile0;                 // first tile (row table index / 128)
    int ntiles, nunits, nA;    // tiles, 16-column units, A stages
    int unit_base;             // first unit of this group in the partial layout
    int d_cols;                // TMEM columns of one accumulator buffer (kDBuf buffers at 0, d_cols, ...)
    int a_col0;                // first TMEM column of the A ring
    int bstage_bytes;          // B_lo bytes per A stage (the singles region of a slot)
    int tile_w[kMaxTiles];
    int dm_col[kMaxTiles];     // TMEM column of tile t's accumulator: [hi*hi | hi*lo + lo*hi] (2W columns)
    int tile_s0[kMaxTiles];    // first single of tile t's window
    int unit_tile[kMaxUnits], unit_c[kMaxUnits];
};

struct Params {
    long ncell, cells_cta;
    int ng, nh, hsep, h_row0;  // maps in the slot; singles; singles from the h part; first h row in a slot
    int slot_bytes, off_b, off_acc, off_bar;
    int s_off, s_chunks;       // singles region of a slot: byte offset and 16-byte chunks (B_lo is made for all)
    int total_units;
    const short2* rows;        // [tiles][128] pairs (j, k); (-1, -1) pads
    double* partial;           // [gridDim.x][total_units][16][128]
    int* err;
    GroupDesc grp[kMaxGroups];
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
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
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

// Non-blocking test of a phase (no suspension): the fast path of the waits below when the phase is already done.
__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait of one thread; false (and the abort flag raised) on timeout or when another role aborted.
__device__ __forceinline__ bool thread_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag, int* err) {
    if (mbar_test(bar, parity)) return true;
    for (unsigned it = 0; it < kSpinLimit; ++it) {
        if (mbar_try(bar, parity)) return true;
        if (*abort_flag) return false;
    }
    *abort_flag = 1;
    atomicExch(err, 1);
    return false;
}
// Bounded wait used while shutting down (no abort check): lets in-flight asynchronous work land.
__device__ __forceinline__ void drain_wait(uint64_t* bar, uint32_t parity, int* err) {
    for (unsigned it = 0; it < kSpinLimit; ++it)
        if (mbar_try(bar, parity)) return;
    atomicExch(err, 1);
}
// Bounded wait of a whole warp with a warp-uniform outcome (the warp then runs .sync.aligned instructions).
__device__ __forceinline__ bool warp_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag, int* err) {
    if (__all_sync(0xffffffffu, mbar_test(bar, parity))) return true;
    for (unsigned it = 0; it < kSpinLimit; ++it) {
        const bool done = mbar_try(bar, parity);
        if (__all_sync(0xffffffffu, done)) return true;
        if (__any_sync(0xffffffffu, *abort_flag != 0)) return false;
    }
    if ((threadIdx.x & 31) == 0) {
        *abort_flag = 1;
        atomicExch(err, 1);
    }
    __syncwarp();
    return false;
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Packed FP32 pairs (two floats in one 64-bit register; sm_100+ f32x2 arithmetic).
__device__ __forceinline__ uint64_t f2pack(float a, float b) {
    return (uint64_t)__float_as_uint(a) | ((uint64_t)__float_as_uint(b) << 32);
}
__device__ __forceinline__ uint64_t mul_x2(uint64_t a, uint64_t b) {
    uint64_t r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ uint64_t sub_x2(uint64_t a, uint64_t b) {
    uint64_t r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
// Two values at once: v = hi + lo with hi = v rounded to TF32 (nearest, ties away from zero: add half a unit of the
// 10-bit mantissa, bit 12, and clear the 13 low bits; a carry moves into the exponent as it should) and lo = v - hi
// in FP32.  lo is symmetric about zero, so the tensor core's truncation of lo to TF32 is unbiased.  (When v is a
// product, the compiler may fuse the multiply into the subtraction; lo then also carries the product's rounding
// error, which only makes hi + lo closer to the exact product.)
__device__ __forceinline__ void split_x2(uint64_t v, uint64_t& hi, uint64_t& lo) {
    const uint32_t h0 = ((uint32_t)v + 0x1000u) & 0xFFFFE000u;
    const uint32_t h1 = ((uint32_t)(v >> 32) + 0x1000u) & 0xFFFFE000u;
    hi = (uint64_t)h0 | ((uint64_t)h1 << 32);
    lo = sub_x2(v, hi);
}

__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t* v) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32};" ::"r"(taddr),
        "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]),
        "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15]), "r"(v[16]), "r"(v[17]), "r"(v[18]),
        "r"(v[19]), "r"(v[20]), "r"(v[21]), "r"(v[22]), "r"(v[23]), "r"(v[24]), "r"(v[25]), "r"(v[26]), "r"(v[27]),
        "r"(v[28]), "r"(v[29]), "r"(v[30]), "r"(v[31]));
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t* v) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr)
        : "memory");
}
// tcgen05.wait::ld tied to two 16-register loads (32 operands).
__device__ __forceinline__ void tmem_wait_ld32(uint32_t* a, uint32_t* b) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(a[0]), "+r"(a[1]), "+r"(a[2]), "+r"(a[3]), "+r"(a[4]), "+r"(a[5]), "+r"(a[6]), "+r"(a[7]),
                   "+r"(a[8]), "+r"(a[9]), "+r"(a[10]), "+r"(a[11]), "+r"(a[12]), "+r"(a[13]), "+r"(a[14]), "+r"(a[15]),
                   "+r"(b[0]), "+r"(b[1]), "+r"(b[2]), "+r"(b[3]), "+r"(b[4]), "+r"(b[5]), "+r"(b[6]), "+r"(b[7]),
                   "+r"(b[8]), "+r"(b[9]), "+r"(b[10]), "+r"(b[11]), "+r"(b[12]), "+r"(b[13]), "+r"(b[14]), "+r"(b[15])
                 :
                 : "memory");
}

// Shared-memory matrix descriptor for the 128-byte swizzle, K-major: 8-row x 128-byte atoms (1024-byte aligned,
// chunk c of row r at r * 128 + ((c ^ (r % 8)) << 4), the layout TMA writes), SBO = 1024 between 8-row groups; the
// K offset within the atom is added to the start address (32 bytes per K = 8 step of TF32).
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)1 << 16;                    // LBO: unused for a swizzled K-major operand
    d |= (uint64_t)(1024 >> 4) << 32;          // SBO
    d |= (uint64_t)1 << 46;                    // descriptor version for tcgen05
    d |= (uint64_t)2 << 61;                    // 128-byte swizzle
    return d;
}

// Instruction descriptor: kind::tf32, D = F32, A = B = TF32, both K-major.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// The MMA and its commit are executed by a whole converged warp and issued by the one lane that elect.sync picks
// (the same lane every time with all 32 active, so the commit tracks the MMAs of the issuing thread).  Keeping the
// issuing code warp-uniform, rather than inside a one-lane branch, lets the compiler hold the operands in uniform
// registers: measured on this part, one thread then issues an M = 128, N = 32 MMA every ~16 cycles (the tensor
// pipe's rate) instead of one every ~200 cycles from a divergent branch.
__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint32_t a_tmem, uint64_t b_desc, uint32_t idesc,
                                         uint32_t accum) {
    asm volatile(
        "{\n\t.reg .pred p, q;\n\telect.sync _|q, 0xffffffff;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "@q tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
        "r"(a_tmem), "l"(b_desc), "r"(idesc), "r"(accum)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile(
        "{\n\t.reg .pred q;\n\telect.sync _|q, 0xffffffff;\n\t"
        "@q tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n\t}" ::"r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
            "r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// 16-byte chunk `ch` (0..7) of map row `r` in a ring slot written by TMA with the 128-byte swizzle: within every
// 1024-byte block the chunk index is XORed with the row index modulo 8.
__device__ __forceinline__ const float4* ring_chunk(const unsigned char* slot, int r, int ch) {
    return reinterpret_cast<const float4*>(slot + r * 128 + ((ch ^ (r & 7)) << 4));
}

// Epilogue of NU output units (a compile-time count keeps the FP32 sums in registers): halfway through every
// period read this warp's TMEM lane quarter of the previous period's accumulators with tcgen05.ld, release the D
// buffer, add into the FP32 sums; every kSpill periods add those into the FP64 sums in shared memory (FP64 is slow
// on this part, so only there); finally write this CTA's FP64 partials.
template <int NU>
__device__ __forceinline__ void epilogue(const GroupDesc& G, const Params& P, uint32_t tmem, double* acc64,
                                         uint64_t* d_full, uint64_t* d_empty, volatile int* abort_flag, int nper,
                                         int warp, int lane) {
    const int q = warp & 3;
    const int row = 32 * q + lane;
    const uint32_t lane_base = (uint32_t)(32 * q) << 16;
    const int ntiles = G.ntiles;
    uint32_t cols[NU][2];     // hi*hi and the corrections (hi*lo + lo*hi) of unit u
#pragma unroll
    for (int u = 0; u < NU; ++u) {
        const int t = G.unit_tile[u], cu = G.unit_c[u];
        cols[u][0] = (uint32_t)(G.dm_col[t] + cu);
        cols[u][1] = (uint32_t)(G.dm_col[t] + G.tile_w[t] + cu);
    }
    const uint32_t d_cols = (uint32_t)G.d_cols;
    int* const err = P.err;
    double* const out = P.partial + ((size_t)blockIdx.x * P.total_units + G.unit_base) * 2048;

    float acc[NU][16];
#pragma unroll
    for (int u = 0; u < NU; ++u)
#pragma unroll
        for (int j = 0; j < 16; ++j) acc[u][j] = 0.f;
    bool ok = true;
    for (int per = 0; per < nper && ok; ++per) {
        const int db = per % kDBuf;
        for (int t = 0; t < ntiles && ok; ++t)
            ok = warp_wait(&d_full[db * kMaxTiles + t], (uint32_t)((per / kDBuf) & 1), abort_flag, err);
        if (!ok) break;
        tc_fence_after();
        const uint32_t dbase = tmem + lane_base + (uint32_t)db * d_cols;
#pragma unroll
        for (int u = 0; u < NU; ++u)
            {
                // both pieces in flight together, one wait
                uint32_t v0[16], v1[16];
                tmem_ld16(dbase + cols[u][0], v0);
                tmem_ld16(dbase + cols[u][1], v1);
                tmem_wait_ld32(v0, v1);
#pragma unroll
                for (int j = 0; j < 16; ++j) acc[u][j] += __uint_as_float(v0[j]) + __uint_as_float(v1[j]);
            }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&d_empty[db]);   // one arrival a warp (the warp's loads are done)
        if ((per + 1) % kSpill == 0) {
#pragma unroll
            for (int u = 0; u < NU; ++u)
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    acc64[(u * 16 + j) * 128 + row] += (double)acc[u][j];
                    acc[u][j] = 0.f;
                }
        }
    }
#pragma unroll
    for (int u = 0; u < NU; ++u)
#pragma unroll
        for (int j = 0; j < 16; ++j) acc64[(u * 16 + j) * 128 + row] += (double)acc[u][j];
    for (int i = 0; i < NU * 16; ++i) out[(size_t)i * 128 + row] = acc64[i * 128 + row];
}


// Producer warp of group gp = (warp - 1) / 4: cells 16 gp .. 16 gp + 15 of every 32-cell stage, for NT tiles (a
// compile-time count: every tile's products live in their own registers, so the next tile's arithmetic does not
// wait for the previous tile's TMEM store to read its registers).  A thread owns TMEM lane 32 (warp % 4) + lane,
// i.e. row `row` of every tile.  The 64 columns of a tile's stage block are [hi 16 | lo 16] of half 0, then of half
// 1; a thread writes its half with one 32-column TMEM store per tile.  (The B operand is made by warp 0.)
template <int NT>
__device__ __forceinline__ void producer(const GroupDesc& G, const Params& P, uint32_t tmem, const unsigned char* ring,
                                         unsigned char* bst, uint64_t* slot_full, uint64_t* slot_empty,
                                         uint64_t* a_full, uint64_t* a_empty, volatile int* abort_flag, int nstages,
                                         int warp, int lane) {
    const int gp = (warp - kProdWarp0) >> 2;
    const int q = warp & 3;
    const int row = 32 * q + lane;
    const uint32_t lane_base = (uint32_t)(32 * q) << 16;
    const int nA = G.nA, a_col0 = G.a_col0, slot_bytes = P.slot_bytes, bstage_bytes = G.bstage_bytes;
    const int s_off = P.s_off, s_chunks = P.s_chunks;
    const int ptid = 32 * (warp - kProdWarp0) + lane;   // 0 .. 255 over both groups
    int* const err = P.err;
    int pj[NT], pk[NT];
#pragma unroll
    for (int t = 0; t < NT; ++t) {
        const short2 jk = P.rows[(size_t)(G.tile0 + t) * 128 + row];
        pj[t] = jk.x;
        pk[t] = jk.y;
    }
    // Rolling prefetch: the operands of the next tile (the next stage's first tile after the last one) are loaded
    // before the current tile's products are formed, so shared-memory latency overlaps the arithmetic.  Padding rows
    // (j < 0) read row 0 and store zeros.
    float4 xc[4], yc[4], xn[4], yn[4];
    uint4 bl[kBloItems];
    // with two tiles warp 3 (idle otherwise) makes B_lo; with one tile the producers have the time for it (one warp
    // would be the slower path: measured), with three warp 3 issues tile 2's MMAs
    constexpr bool kBloByProducers = NT != 2;
    auto load_tile = [&](const unsigned char* slot, int t, float4 (&x)[4], float4 (&y)[4]) {
        const int j = max(pj[t], 0), k = max(pk[t], 0);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            x[c] = *ring_chunk(slot, j, 4 * gp + c);
            y[c] = *ring_chunk(slot, k, 4 * gp + c);
        }
    };
    auto load_blo = [&](const unsigned char* slot, uint4 (&b)[kBloItems]) {
#pragma unroll
        for (int m = 0; m < kBloItems; ++m)
            if (ptid + 256 * m < s_chunks) b[m] = *reinterpret_cast<const uint4*>(slot + s_off + 16 * (ptid + 256 * m));
    };
    // tensor-memory addresses from warp-uniform, divide-free values (the base is 0: the CTA holds all 512
    // columns; the issuing warps check it), so that the compiler keeps the store addresses in uniform registers
    if (nstages <= 0 || tmem != 0u) return;
    if (!warp_wait(&slot_full[0], 0u, abort_flag, err)) return;
    load_tile(ring, 0, xc, yc);
    if (kBloByProducers) load_blo(ring, bl);
    int s = 0, as = 0, s1 = 1 % kRingSlots;
    uint32_t aph = 1u, s1ph = 0u;                        // a_empty parity of round st / nA - 1; slot_full of st + 1
    uint32_t a_stage = (uint32_t)a_col0;
    const uint32_t a_step = 64u * NT;
    for (int st = 0; st < nstages; ++st) {
        const unsigned char* slot = ring + (size_t)s * slot_bytes;
        bool ok = true;
#pragma unroll
        for (int t = 0; t < NT; ++t) {
            // (no break inside this unrolled loop: a failed wait clears ok, the rest of the stage is skipped)
            if (t + 1 < NT) {
                load_tile(slot, t + 1, xn, yn);
            } else if (st + 1 < nstages) {
                ok = ok && warp_wait(&slot_full[s1], s1ph, abort_flag, err);
                if (ok) load_tile(ring + (size_t)s1 * slot_bytes, 0, xn, yn);
            }
            if (t == 0) {
                // tensor memory A stage and B_lo stage `as` are free once the MMAs of stage st - nA completed
                if (st >= nA) ok = ok && warp_wait(&a_empty[as], aph, abort_flag, err);
                tc_fence_after();
            }
            if (!ok) continue;
            uint32_t v[32];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                uint64_t h0, l0, h1, l1;
                split_x2(mul_x2(f2pack(xc[c].x, xc[c].y), f2pack(yc[c].x, yc[c].y)), h0, l0);
                split_x2(mul_x2(f2pack(xc[c].z, xc[c].w), f2pack(yc[c].z, yc[c].w)), h1, l1);
                v[4 * c + 0] = (uint32_t)h0;
                v[4 * c + 1] = (uint32_t)(h0 >> 32);
                v[4 * c + 2] = (uint32_t)h1;
                v[4 * c + 3] = (uint32_t)(h1 >> 32);
                v[16 + 4 * c + 0] = (uint32_t)l0;
                v[16 + 4 * c + 1] = (uint32_t)(l0 >> 32);
                v[16 + 4 * c + 2] = (uint32_t)l1;
                v[16 + 4 * c + 3] = (uint32_t)(l1 >> 32);
            }
            if (pj[t] < 0) {
#pragma unroll
                for (int c = 0; c < 32; ++c) v[c] = 0u;
            }
            tmem_st32(lane_base + a_stage + (uint32_t)(64 * t + 32 * gp), v);
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                xc[c] = xn[c];
                yc[c] = yn[c];
            }
        }
        if (!ok) break;
        // B_lo = (g - trunc(g)) rounded to TF32 (nearest, ties away), at the same byte offset as g (same swizzle)
        unsigned char* bs = bst + (size_t)as * bstage_bytes;
#pragma unroll
        for (int m = 0; m < kBloItems; ++m) {
            if (kBloByProducers && ptid + 256 * m < s_chunks) {
                uint32_t* w = reinterpret_cast<uint32_t*>(&bl[m]);
                const uint64_t g01 = (uint64_t)w[0] | ((uint64_t)w[1] << 32);
                const uint64_t g23 = (uint64_t)w[2] | ((uint64_t)w[3] << 32);
                const uint64_t t01 = g01 & 0xFFFFE000FFFFE000ull, t23 = g23 & 0xFFFFE000FFFFE000ull;
                const uint64_t l01 = sub_x2(g01, t01), l23 = sub_x2(g23, t23);
                *reinterpret_cast<uint4*>(bs + 16 * (ptid + 256 * m)) =
                    make_uint4(((uint32_t)l01 + 0x1000u) & 0xFFFFE000u, ((uint32_t)(l01 >> 32) + 0x1000u) & 0xFFFFE000u,
                               ((uint32_t)l23 + 0x1000u) & 0xFFFFE000u, ((uint32_t)(l23 >> 32) + 0x1000u) & 0xFFFFE000u);
            }
        }
        // the next stage's B_lo chunks (its slot is already full: waited for the first tile's prefetch)
        if (kBloByProducers && st + 1 < nstages) load_blo(ring + (size_t)s1 * slot_bytes, bl);
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // B_lo stores -> tensor core
        tc_fence_before();
        // one arrival a warp on each barrier: __syncwarp orders the other lanes' stores and reads before lane 0's
        // release (256 single-thread arrivals were 512 shared-memory atomics on two words every stage)
        __syncwarp();
        if (lane == 0) {
            mbar_arrive(&a_full[as]);
            mbar_arrive(&slot_empty[s]);
        }
        s = s1;
        if (++s1 == kRingSlots) { s1 = 0; s1ph ^= 1u; }
        if (++as == nA) { as = 0; aph ^= 1u; a_stage = (uint32_t)a_col0; } else { a_stage += a_step; }
    }
}

__global__ void __launch_bounds__(kThreads, 1)
    k_contract_tc(const __grid_constant__ CUtensorMap tmap_g, const __grid_constant__ CUtensorMap tmap_h,
                  const __grid_constant__ Params P) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    const GroupDesc& G = P.grp[blockIdx.y];
    unsigned char* ring = smem;
    unsigned char* bst = smem + P.off_b;
    double* acc64 = reinterpret_cast<double*>(smem + P.off_acc);                 // [unit][16][128]
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + P.off_bar);
    uint64_t* slot_full = bars;                        // [kRingSlots]  TMA -> producers
    uint64_t* slot_empty = bars + kRingSlots;          // [kRingSlots]  producers -> TMA
    uint64_t* a_full = bars + 2 * kRingSlots;          // [kMaxAStages] producers -> issuers
    uint64_t* a_empty = a_full + kMaxAStages;          // [kMaxAStages] MMA commit -> producers
    uint64_t* d_full = a_empty + kMaxAStages;          // [2][kMaxTiles] MMA commit -> epilogue (D buffer, tile)
    uint64_t* d_empty = d_full + 2 * kMaxTiles;        // [2]            epilogue -> issuers (D buffer)
    uint64_t* fin = d_empty + 2;                       // [kMaxTiles]
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(fin + kMaxTiles);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

    // warp index through a shuffle from lane 0: the compiler then knows it is warp-uniform, so role branches and
    // the tensor-memory addresses derived from it stay in uniform registers
    const int tid = threadIdx.x, lane = tid & 31;
    const int warp = __shfl_sync(0xffffffffu, tid >> 5, 0);
    const long c0 = (long)blockIdx.x * P.cells_cta;
    const long c1 = min(P.ncell, c0 + P.cells_cta);
    const int nslots = c0 < c1 ? (int)((c1 - c0 + kSlotCells - 1) / kSlotCells) : 0;
    const int nstages = nslots;                 // one A stage per ring slot
    // plan fields used in the loops, in registers
    const int nA = G.nA, ntiles = G.ntiles, a_col0 = G.a_col0, bstage_bytes = G.bstage_bytes;
    const int slot_bytes = P.slot_bytes;
    int* const err = P.err;

    for (int i = tid; i < G.nunits * 16 * 128; i += kThreads) acc64[i] = 0.0;
    if (tid == 0) {
        for (int s = 0; s < kRingSlots; ++s) {
            mbar_init(&slot_full[s], 1);
            // producer warps read a slot, the MMAs read B_hi, warp 3 (two tiles) reads it for B_lo
            mbar_init(&slot_empty[s], kProdWarps + ntiles + (ntiles == 2 ? 1 : 0));
        }
        for (int s = 0; s < kMaxAStages; ++s) {
            // both producer groups make a stage's A (and B_lo, except with two tiles: then warp 3 makes it)
            mbar_init(&a_full[s], kProdWarps + (ntiles == 2 ? 1 : 0));
            mbar_init(&a_empty[s], ntiles);        // one commit per issuing thread (tile)
        }
        for (int i = 0; i < 2 * kMaxTiles; ++i) mbar_init(&d_full[i], 1);
        for (int i = 0; i < 2; ++i) mbar_init(&d_empty[i], kEpiWarps);
        for (int i = 0; i < kMaxTiles; ++i) mbar_init(&fin[i], 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(tmem_slot)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp < kProdWarp0) {
        // warpgroup 0 hands registers to the producers (all four warps, one instruction)
        asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(kRegsCtl));
        if (warp == 0) {
            // ------------------------------------------------------------------ TMA producer
            if (lane == 0 && nslots > 0) {
                const uint32_t bytes = (uint32_t)(P.ng * 128 + (P.hsep ? P.nh * 128 : 0));
                const bool hsep = P.hsep != 0;
                const int hoff = P.h_row0 * 128;
                int issued = 0;
                for (int sl = 0; sl < nslots; ++sl) {
                    const int s = sl % kRingSlots;
                    if (sl >= kRingSlots &&
                        !thread_wait(&slot_empty[s], (uint32_t)((sl / kRingSlots - 1) & 1), abort_flag, err))
                        break;
                    unsigned char* dst = ring + (size_t)s * slot_bytes;
                    const int x = (int)(c0 + (long)sl * kSlotCells);
                    mbar_expect_tx(&slot_full[s], bytes);
                    tma_load_2d(dst, &tmap_g, x, 0, &slot_full[s]);
                    if (hsep) tma_load_2d(dst + hoff, &tmap_h, x, 0, &slot_full[s]);
                    ++issued;
                }
                // every load issued has landed before the CTA may exit
                for (int sl = max(0, issued - kRingSlots); sl < issued; ++sl)
                    drain_wait(&slot_full[sl % kRingSlots], (uint32_t)((sl / kRingSlots) & 1), err);
            }
            __syncwarp();
        } else if (warp == 3 && ntiles == 2) {
            // ------------------------------------------------------------------ B_lo (two tiles)
            // every 16-byte chunk of a slot's singles region -> (g - trunc(g)) rounded to TF32, same offset in the
            // B_lo stage; released to the issuers with one arrival on the stage barrier
            const int s_off = P.s_off, s_chunks = P.s_chunks;
            int s = 0, as = 0;
            uint32_t sph = 0u, aph = 1u;
            for (int st = 0; st < nstages; ++st) {
                if (!warp_wait(&slot_full[s], sph, abort_flag, err)) break;
                if (st >= nA && !warp_wait(&a_empty[as], aph, abort_flag, err)) break;
                const unsigned char* src = ring + (size_t)s * slot_bytes + s_off;
                unsigned char* dst = bst + (size_t)as * bstage_bytes;
                for (int i0 = 0; i0 < s_chunks; i0 += 128) {
                    uint4 g[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int i = i0 + 32 * u + lane;
                        if (i < s_chunks) g[u] = *reinterpret_cast<const uint4*>(src + 16 * i);
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int i = i0 + 32 * u + lane;
                        if (i < s_chunks) {
                            const uint64_t g01 = (uint64_t)g[u].x | ((uint64_t)g[u].y << 32);
                            const uint64_t g23 = (uint64_t)g[u].z | ((uint64_t)g[u].w << 32);
                            const uint64_t l01 = sub_x2(g01, g01 & 0xFFFFE000FFFFE000ull);
                            const uint64_t l23 = sub_x2(g23, g23 & 0xFFFFE000FFFFE000ull);
                            *reinterpret_cast<uint4*>(dst + 16 * i) = make_uint4(
                                ((uint32_t)l01 + 0x1000u) & 0xFFFFE000u, ((uint32_t)(l01 >> 32) + 0x1000u) & 0xFFFFE000u,
                                ((uint32_t)l23 + 0x1000u) & 0xFFFFE000u, ((uint32_t)(l23 >> 32) + 0x1000u) & 0xFFFFE000u);
                        }
                    }
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // B_lo stores -> tensor core
                __syncwarp();
                if (lane == 0) {
                    mbar_arrive(&a_full[as]);
                    mbar_arrive(&slot_empty[s]);
                }
                if (++s == kRingSlots) { s = 0; sph ^= 1u; }
                if (++as == nA) { as = 0; aph ^= 1u; }
            }
        } else if (warp - 1 < ntiles) {
            // ------------------------------------------------------------------ MMA issue (warp 1 + t: tile t)
            // The whole warp runs the loop (converged; every lane polls the barriers); the elected lane issues and
            // commits inside mma_tf32 / mma_commit.
            // tile t's window of singles: rows s0 .. s0 + W - 1 of a slot's singles region (B_hi: the slot itself, read
            // as TF32, i.e. truncated) and of the B_lo stage (same layout)
            const uint32_t ring_s = smem_u32(ring) + (uint32_t)P.s_off, bst_s = smem_u32(bst);
            const int t = warp - 1;
            const int W = G.tile_w[t];
            const uint32_t idesc_w = idesc_tf32(128, W);
            // Every operand below is built from warp-uniform values (parameters, constants, loop-carried counters;
            // no division) so that the compiler keeps it in uniform registers: the tensor memory base is the
            // constant 0, which is what a CTA allocating all 512 columns receives (lane 0, column 0).
            const bool tmem_ok = tmem == 0u;
            if (!tmem_ok && lane == 0) {
                *abort_flag = 1;
                atomicExch(err, 1);
            }
            const uint32_t dm = (uint32_t)G.dm_col[t], dc = dm + (uint32_t)W;
            const uint32_t a_first = (uint32_t)(a_col0 + 64 * t), a_step = (uint32_t)(64 * ntiles);
            const uint64_t bh_first = sdesc_sw128(ring_s + (uint32_t)(128 * G.tile_s0[t]));
            const uint64_t bl_first = sdesc_sw128(bst_s + (uint32_t)(128 * G.tile_s0[t]));
            // descriptor address steps (16-byte units; no carry out of the 14-bit field: shared memory < 2^18 bytes)
            const uint64_t bh_step = (uint64_t)(slot_bytes >> 4), bl_step = (uint64_t)(bstage_bytes >> 4);
            int s = 0, as = 0, pos = 0, per = 0;
            uint32_t sph = 0, aph = 0;
            uint32_t aa = a_first;
            uint64_t bh = bh_first, bl = bl_first;
            for (int st = 0; st < nstages && tmem_ok; ++st) {
                const bool pstart = pos == 0;
                // one accumulator buffer: a period's first MMAs wait until the epilogue has read the previous one
                if (pstart && per >= 1 && !warp_wait(&d_empty[0], (uint32_t)((per - 1) & 1), abort_flag, err)) break;
                if (!warp_wait(&slot_full[s], sph, abort_flag, err)) break;
                if (!warp_wait(&a_full[as], aph, abort_flag, err)) break;
                tc_fence_after();
#pragma unroll
                for (int ks = 0; ks < kKC / 8; ++ks) {
                    // K step ks: cells 8 ks .. 8 ks + 7; A_hi at half (ks / 2), column 8 (ks % 2); A_lo at +16.  B
                    // advances 32 bytes a step within the swizzle atom (2 in the descriptor's address field)
                    const uint32_t ah = aa + 32u * (ks >> 1) + 8u * (ks & 1);
                    const uint32_t acc = (pstart && ks == 0) ? 0u : 1u;
                    mma_tf32(dm, ah, bh + (uint64_t)(2 * ks), idesc_w, acc);          // A_hi . B_hi
                    mma_tf32(dc, ah, bl + (uint64_t)(2 * ks), idesc_w, acc);          // A_hi . B_lo
                    mma_tf32(dc, ah + 16u, bh + (uint64_t)(2 * ks), idesc_w, 1u);     // + A_lo . B_hi
                }
                mma_commit(&a_empty[as]);
                mma_commit(&slot_empty[s]);
                if (pos == kPeriod - 1 || st == nstages - 1) mma_commit(&d_full[t]);
                if (++s == kRingSlots) { s = 0; sph ^= 1u; bh = bh_first; } else { bh += bh_step; }
                if (++as == nA) { as = 0; aph ^= 1u; aa = a_first; bl = bl_first; } else { aa += a_step; bl += bl_step; }
                if (++pos == kPeriod) { pos = 0; ++per; }
            }
            // every MMA issued by the elected thread has completed before TMEM is released
            mma_commit(&fin[t]);
            drain_wait(&fin[t], 0, err);
            __syncwarp();
        }
    } else if (warp < kProdWarp0 + kProdWarps) {
        asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(kRegsProd));
        // ------------------------------------------------------------------ producers
        switch (ntiles) {
            case 1: producer<1>(G, P, tmem, ring, bst, slot_full, slot_empty, a_full, a_empty, abort_flag, nstages, warp, lane); break;
            case 2: producer<2>(G, P, tmem, ring, bst, slot_full, slot_empty, a_full, a_empty, abort_flag, nstages, warp, lane); break;
            default: producer<3>(G, P, tmem, ring, bst, slot_full, slot_empty, a_full, a_empty, abort_flag, nstages, warp, lane); break;
        }
    } else {
        // ------------------------------------------------------------------ epilogue
        const int nper = (nstages + kPeriod - 1) / kPeriod;
        switch (G.nunits) {
            case 1: epilogue<1>(G, P, tmem, acc64, d_full, d_empty, abort_flag, nper, warp, lane); break;
            case 2: epilogue<2>(G, P, tmem, acc64, d_full, d_empty, abort_flag, nper, warp, lane); break;
            default: epilogue<3>(G, P, tmem, acc64, d_full, d_empty, abort_flag, nper, warp, lane); break;
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem));
}

// out[o] = sum over CTAs of partial[cta][gidx[o]], in CTA order (deterministic).
__global__ void k_reduce_gather(const double* __restrict__ partial, int ncta, long stride,
                                const int* __restrict__ gidx, int n_out, double* __restrict__ out) {
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= n_out) return;
    const long g = gidx[o];
    double s = 0.0;
    for (int c = 0; c < ncta; ++c) s += partial[(long)c * stride + g];
    out[o] = s;
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

// ------------------------------------------------------------------------------------------------ self-check
// What the split-TF32 scheme assumes of the tensor core, checked on known operands: an FP32 B operand is read as TF32
// by dropping its 13 low bits (B_hi = the raw map), and a TF32 value written to tensor memory as the A operand is
// used exactly.  A (tensor memory, M = 128, K = 8) has A[0][0] = 1 and A[1][0] = 1 + 2^-10; B (shared memory, N = 16,
// 128-byte swizzle) has B[0][0] = 1 + 3 2^-12, three quarters of a TF32 unit above 1.  Truncation gives D[0][0] = 1
// and D[1][0] = 1 + 2^-10; rounding to nearest would give 1 + 2^-10 and (1 + 2^-10)^2.  res: D[0][0], D[1][0] (FP32
// bit patterns) and a timeout flag.
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t* v) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(taddr), "r"(v[0]),
                 "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]));
}

__global__ void __launch_bounds__(128, 1) k_tf32_selfcheck(uint32_t* res) {
    __shared__ __align__(1024) unsigned char sB[16 * 128];
    __shared__ uint64_t bar;
    __shared__ uint32_t tslot;
    const int tid = threadIdx.x, lane = tid & 31;
    const int warp = __shfl_sync(0xffffffffu, tid >> 5, 0);
    for (int i = tid; i < 16 * 128 / 4; i += 128) reinterpret_cast<uint32_t*>(sB)[i] = 0u;
    if (tid == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 32;" ::"r"(smem_u32(&tslot)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    __syncthreads();
    if (tid == 0) reinterpret_cast<float*>(sB)[0] = 1.0f + 3.0f * 0x1p-12f;   // row 0, chunk 0 (unswizzled position)
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tslot;
    {
        const int r = 32 * warp + lane;                  // TMEM lane of this thread
        uint32_t v[8] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
        if (r == 0) v[0] = __float_as_uint(1.0f);
        if (r == 1) v[0] = __float_as_uint(1.0f + 0x1p-10f);
        tmem_st8(tmem + ((uint32_t)(32 * warp) << 16), v);
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) {
        mma_tf32(tmem + 8u, tmem, sdesc_sw128(smem_u32(sB)), idesc_tf32(128, 16), 0u);
        mma_commit(&bar);
        unsigned it = 0;
        for (; it < (1u << 20); ++it)
            if (mbar_try(&bar, 0)) break;
        if (lane == 0) res[2] = it == (1u << 20) ? 1u : 0u;
        tc_fence_after();
        uint32_t d[16];
        tmem_ld16(tmem + 8u, d);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (lane < 2) res[lane] = d[0];
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 32;" ::"r"(tmem));
}

// ------------------------------------------------------------------------------------------------ Gram
// Tensor-core Gram matrix of the bispectrum Fisher (Sec. 4.3.4, eq. bk-fish-def in Fourier space):
//   part[s][i][j] = sum_{k in split s} A[i][k] B[j][k],  A = Z (weighted), B = Y as float32 rows [n][K], K = 2 M
// (real and imaginary parts of the binned modes interleaved: re*re + im*im is the real part of conj(Z) Y).
// A CTA takes a 128 x 32 output tile and a contiguous range of K.  Arithmetic as in the triplet contraction:
// A = A_hi + A_lo (A_hi rounded to TF32 by the producers, written to tensor memory), B_hi = the raw TMA tile (read as
// TF32 by truncation), B_lo = (B - trunc B) rounded to TF32; D_hh += A_hi B_hi, D_c += A_hi B_lo + A_lo B_hi; D restarts
// every 64 K (8 MMAs a column), FP32 register sums, FP64 register sums every 2048 K; FP64 partials per K split.
namespace gram {
constexpr int kBM = 128, kBN = 32, kKC = 32, kStages = 6, kPeriod = 2, kSpill = 32;
constexpr int kThreads = 384;   // warps 0 TMA/TMEM, 1 MMA, 2 B_lo, 3 idle, 4-7 A producers, 8-11 epilogue
constexpr int kAStage = kBM * 128, kBStage = kBN * 128;   // raw tiles: 32 floats (128 B) a row
constexpr int kSmem = kStages * (kAStage + 2 * kBStage) + 1024 + 256;

struct GP {
    long k_cta;       // K per CTA (multiple of kKC)
    long K;           // row length (floats)
    int nA, nB, nsplit;
    double* part;     // [nsplit][nI*128][nJ*32]
    long ldp;         // row stride of part (nJ * 32)
    long split_stride;
    int* err;
};

__global__ void __launch_bounds__(kThreads, 1)
    k_gram_tc(const __grid_constant__ CUtensorMap tA, const __grid_constant__ CUtensorMap tB, const __grid_constant__ GP P) {
    extern __shared__ __align__(1024) unsigned char gsm_raw[];
    unsigned char* sm = gsm_raw + ((1024u - (smem_u32(gsm_raw) & 1023u)) & 1023u);
    unsigned char* sA = sm;                                       // [kStages][kAStage]
    unsigned char* sB = sA + kStages * kAStage;                   // [kStages][kBStage]
    unsigned char* sBl = sB + kStages * kBStage;                  // [kStages][kBStage]
    uint64_t* bars = reinterpret_cast<uint64_t*>(sBl + kStages * kBStage);
    uint64_t* full = bars;                      // [kStages] TMA -> A producers, B_lo warp
    uint64_t* ready = full + kStages;           // [kStages] A producers + B_lo -> MMA
    uint64_t* empty = ready + kStages;          // [kStages] MMA commit -> TMA
    uint64_t* d_full = empty + kStages;         // MMA -> epilogue (period done)
    uint64_t* d_empty = d_full + 1;             // epilogue -> MMA
    uint64_t* fin = d_empty + 1;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(fin + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

    const int tid = threadIdx.x, lane = tid & 31;
    const int warp = __shfl_sync(0xffffffffu, tid >> 5, 0);
    const int i0 = blockIdx.y * kBM, j0 = blockIdx.x * kBN;
    const long k0 = (long)blockIdx.z * P.k_cta;
    const long k1 = min(P.K, k0 + P.k_cta);
    const int nst = k0 < k1 ? (int)((k1 - k0 + kKC - 1) / kKC) : 0;
    int* const err = P.err;
    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&ready[s], 5);
            mbar_init(&empty[s], 1);
        }
        mbar_init(d_full, 1);
        mbar_init(d_empty, 4);
        mbar_init(fin, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(tmem_slot)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    // TMEM columns: D_hh [0, 32), D_c [32, 64), A stage s: hi [64 + 64 s, +32), lo [+32, +64)
    if (warp == 0) {
        if (lane == 0 && nst > 0) {
            int issued = 0;
            for (int st = 0; st < nst; ++st) {
                const int s = st % kStages;
                if (st >= kStages && !thread_wait(&empty[s], (uint32_t)((st / kStages - 1) & 1), abort_flag, err)) break;
                const int x = (int)(k0 + (long)st * kKC);
                mbar_expect_tx(&full[s], (uint32_t)(kAStage + kBStage));
                tma_load_2d(sA + (size_t)s * kAStage, &tA, x, i0, &full[s]);
                tma_load_2d(sB + (size_t)s * kBStage, &tB, x, j0, &full[s]);
                ++issued;
            }
            for (int st = max(0, issued - kStages); st < issued; ++st)
                drain_wait(&full[st % kStages], (uint32_t)((st / kStages) & 1), err);
        }
        __syncwarp();
    } else if (warp == 1) {
        // MMA issue (whole warp converged; the elected lane issues)
        const bool tmem_ok = tmem == 0u;
        if (!tmem_ok && lane == 0) { *abort_flag = 1; atomicExch(err, 1); }
        const uint32_t idesc = idesc_tf32(kBM, kBN);
        const uint64_t bh0 = sdesc_sw128(smem_u32(sB)), bl0 = sdesc_sw128(smem_u32(sBl));
        const uint64_t bstep = (uint64_t)(kBStage >> 4);
        int s = 0, pos = 0, per = 0;
        uint32_t ph = 0;
        uint32_t aa = 64u;
        uint64_t bh = bh0, bl = bl0;
        for (int st = 0; st < nst && tmem_ok; ++st) {
            const bool pstart = pos == 0;
            if (pstart && per >= 1 && !warp_wait(d_empty, (uint32_t)((per - 1) & 1), abort_flag, err)) break;
            if (!warp_wait(&ready[s], ph, abort_flag, err)) break;
            tc_fence_after();
#pragma unroll
            for (int ks = 0; ks < kKC / 8; ++ks) {
                const uint32_t acc = (pstart && ks == 0) ? 0u : 1u;
                mma_tf32(0u, aa + 8u * ks, bh + (uint64_t)(2 * ks), idesc, acc);          // A_hi B_hi
                mma_tf32(32u, aa + 8u * ks, bl + (uint64_t)(2 * ks), idesc, acc);         // A_hi B_lo
                mma_tf32(32u, aa + 32u + 8u * ks, bh + (uint64_t)(2 * ks), idesc, 1u);    // + A_lo B_hi
            }
            mma_commit(&empty[s]);
            if (pos == kPeriod - 1 || st == nst - 1) mma_commit(d_full);
            if (++s == kStages) { s = 0; ph ^= 1u; aa = 64u; bh = bh0; bl = bl0; } else { aa += 64u; bh += bstep; bl += bstep; }
            if (++pos == kPeriod) { pos = 0; ++per; }
        }
        mma_commit(fin);
        drain_wait(fin, 0, err);
        __syncwarp();
    } else if (warp == 2) {
        // B_lo = (B - trunc B) rounded to TF32, same swizzled layout: 32 rows x 8 chunks, 8 chunks a lane
        int s = 0;
        uint32_t ph = 0;
        for (int st = 0; st < nst; ++st) {
            if (!warp_wait(&full[s], ph, abort_flag, err)) break;
            const unsigned char* src = sB + (size_t)s * kBStage;
            unsigned char* dst = sBl + (size_t)s * kBStage;
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int i = lane + 32 * u;
                const uint4 g = *reinterpret_cast<const uint4*>(src + 16 * i);
                const uint64_t g01 = (uint64_t)g.x | ((uint64_t)g.y << 32);
                const uint64_t g23 = (uint64_t)g.z | ((uint64_t)g.w << 32);
                const uint64_t l01 = sub_x2(g01, g01 & 0xFFFFE000FFFFE000ull);
                const uint64_t l23 = sub_x2(g23, g23 & 0xFFFFE000FFFFE000ull);
                *reinterpret_cast<uint4*>(dst + 16 * i) =
                    make_uint4(((uint32_t)l01 + 0x1000u) & 0xFFFFE000u, ((uint32_t)(l01 >> 32) + 0x1000u) & 0xFFFFE000u,
                               ((uint32_t)l23 + 0x1000u) & 0xFFFFE000u, ((uint32_t)(l23 >> 32) + 0x1000u) & 0xFFFFE000u);
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(&ready[s]);
            if (++s == kStages) { s = 0; ph ^= 1u; }
        }
    } else if (warp >= 4 && warp < 8) {
        // A producers: thread = row r = 32 (warp % 4) + lane of the tile = TMEM lane r; hi / lo of the 32 K values
        const int q = warp & 3, r = 32 * q + lane;
        const uint32_t lane_base = (uint32_t)(32 * q) << 16;
        if (tmem == 0u) {
            int s = 0;
            uint32_t ph = 0;
            uint32_t ac = 64u;
            for (int st = 0; st < nst; ++st) {
                if (!warp_wait(&full[s], ph, abort_flag, err)) break;
                const unsigned char* row = sA + (size_t)s * kAStage;
                uint32_t v[32], w[32];
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    const float4 x = *ring_chunk(row, r, c);
                    uint64_t h0, l0, h1, l1;
                    split_x2(f2pack(x.x, x.y), h0, l0);
                    split_x2(f2pack(x.z, x.w), h1, l1);
                    v[4 * c + 0] = (uint32_t)h0; v[4 * c + 1] = (uint32_t)(h0 >> 32);
                    v[4 * c + 2] = (uint32_t)h1; v[4 * c + 3] = (uint32_t)(h1 >> 32);
                    w[4 * c + 0] = (uint32_t)l0; w[4 * c + 1] = (uint32_t)(l0 >> 32);
                    w[4 * c + 2] = (uint32_t)l1; w[4 * c + 3] = (uint32_t)(l1 >> 32);
                }
                tmem_st32(lane_base + ac, v);
                tmem_st32(lane_base + ac + 32u, w);
                asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&ready[s]);
                if (++s == kStages) { s = 0; ph ^= 1u; ac = 64u; } else { ac += 64u; }
            }
        }
    } else if (warp >= 8) {
        // epilogue: lane r of the tile; every period add D_hh + D_c into FP32 sums, every kSpill periods into FP64
        const int q = warp & 3, r = 32 * q + lane;
        const uint32_t lane_base = (uint32_t)(32 * q) << 16;
        const int nper = (nst + kPeriod - 1) / kPeriod;
        float acc[kBN];
        double acc64[kBN];
#pragma unroll
        for (int j = 0; j < kBN; ++j) { acc[j] = 0.f; acc64[j] = 0.0; }
        for (int per = 0; per < nper; ++per) {
            if (!warp_wait(d_full, (uint32_t)(per & 1), abort_flag, err)) break;
            tc_fence_after();
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                uint32_t a[16], b[16];
                tmem_ld16(tmem + lane_base + 16u * h, a);
                tmem_ld16(tmem + lane_base + 32u + 16u * h, b);
                tmem_wait_ld32(a, b);
#pragma unroll
                for (int j = 0; j < 16; ++j) acc[16 * h + j] += __uint_as_float(a[j]) + __uint_as_float(b[j]);
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(d_empty);
            if ((per + 1) % kSpill == 0) {
#pragma unroll
                for (int j = 0; j < kBN; ++j) { acc64[j] += (double)acc[j]; acc[j] = 0.f; }
            }
        }
        double* out = P.part + (size_t)blockIdx.z * P.split_stride + (size_t)(i0 + r) * P.ldp + j0;
#pragma unroll
        for (int j = 0; j < kBN; ++j) out[j] = acc64[j] + (double)acc[j];
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem));
}

// out[i][j] += scale * sum_s part[s][i][j] (splits in order), i < nA, j < nB.
__global__ void k_gram_reduce(const double* __restrict__ part, int nsplit, long split_stride, long ldp, int nA, int nB,
                              double scale, double* __restrict__ out) {
    const long o = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= (long)nA * nB) return;
    const int i = (int)(o / nB), j = (int)(o - (long)i * nB);
    double s = 0.0;
    for (int q = 0; q < nsplit; ++q) s += part[(size_t)q * split_stride + (size_t)i * ldp + j];
    out[o] += scale * s;
}
}  // namespace gram

// ------------------------------------------------------------------------------------------------ host planner

// A pair row with the range of singles it needs and where each of its outputs goes.
struct NeedPair {
    int j, k;
    int lo, hi;                                   // singles needed: [lo, hi]
    std::vector<std::pair<int, int>> outs;        // (single, output index)
};

// Run-time choices of a plan that leave the kernel unchanged, tried by the autotuner: the per-tile cost of the
// tile-cutting DP (small: more, narrower tiles; large: fewer, wider ones), the number of tiles a row group (CTA)
// may take, and the cell split (0: one CTA per SM and row group, ngroups waves; 1: one wave of SMs / ngroups CTAs
// per group; 2: two CTAs per SM and row group, shorter cell ranges).
struct PlanOpts {
    int tile_cost = 8;
    int group_cap = 3;
    int cta_mode = 0;
};

struct Plan {
    int ng = 0, nh = 0, hsep = 0, n_out = 0, ncta = 0, ngroups = 0, total_units = 0;
    PlanOpts opts{};
    bool tuned = false;
    float tuned_ms = 0.f;   // time of the chosen candidate (0 when not tuned)
    int tuned_of = 0;       // candidates timed
    // what the plan was built from (the autotuner rebuilds it with other options)
    std::vector<NeedPair> need;
    int sing_g = 0;
    long ncell = 0;
    long cells_cta = 0;
    Params base{};
    size_t smem = 0;
    short2* d_rows = nullptr;
    int* d_gidx = nullptr;
    double* d_partial = nullptr;
    ~Plan() {
        if (d_rows) cudaFree(d_rows);
        if (d_gidx) cudaFree(d_gidx);
        if (d_partial) cudaFree(d_partial);
    }
};

static int round_w(int w) { return w <= 16 ? 16 : 32; }

// Tiles of <= 128 pairs, consecutive in the order of (hi, lo), cut by dynamic programming to minimise the summed
// window width (the tensor work) plus a per-tile cost.
static std::vector<std::pair<int, int>> cut_tiles(const std::vector<NeedPair>& P, int tile_cost) {
    const int n = (int)P.size();
    std::vector<long> f(n + 1, (long)1 << 40);
    std::vector<int> arg(n + 1, 0);
    f[0] = 0;
    for (int i = 1; i <= n; ++i) {
        int lo = 1 << 30, hi = -1;
        for (int j = i - 1; j >= 0 && j >= i - 128; --j) {
            lo = std::min(lo, P[j].lo);
            hi = std::max(hi, P[j].hi);
            const int s0 = lo / 8 * 8;
            if (hi + 1 - s0 > 32) break;
            const long c = f[j] + round_w(hi + 1 - s0) + tile_cost;
            if (c < f[i]) { f[i] = c; arg[i] = j; }
        }
    }
    std::vector<std::pair<int, int>> seg;
    for (int i = n; i > 0; i = arg[i]) seg.push_back({arg[i], i});
    std::reverse(seg.begin(), seg.end());
    return seg;
}

// Pure host layout of a plan (no CUDA calls): tiles, row groups, TMEM / shared-memory layout, the row table and the
// gather index of every output.  Returns nullptr or an error message.
// sing_g = 1 with hsep = 1: the slot holds the g rows and the h rows (pairs may take one map from each, h rows at
// index h_row0 + i) and the singles are the g rows.
static const char* layout_plan(Plan& pl, long ncell, int nsm, int ng, int nh, int hsep, std::vector<NeedPair> need,
                               int n_out, std::vector<short2>& rows, std::vector<int>& gidx, int sing_g = 0,
                               const PlanOpts& opts = PlanOpts{}) {
    pl.ng = ng; pl.nh = nh; pl.hsep = hsep; pl.n_out = n_out;
    pl.opts = opts;
    if (opts.group_cap < 1 || opts.group_cap > kMaxTiles || opts.cta_mode < 0 || opts.cta_mode > 2)
        return "contract_tc: bad plan options";
    std::stable_sort(need.begin(), need.end(), [](const NeedPair& a, const NeedPair& b) {
        return std::tie(a.hi, a.lo) < std::tie(b.hi, b.lo);
    });
    for (const NeedPair& p : need)
        if (p.hi + 1 - p.lo / 8 * 8 > 32) return "contract_tc: a pair needs a window of more than 32 singles";
    auto seg = need.empty() ? std::vector<std::pair<int, int>>{} : cut_tiles(need, opts.tile_cost);
    struct TileH { int first, last, s0, W; };
    std::vector<TileH> tiles;
    for (auto& sg : seg) {
        int lo = 1 << 30, hi = -1;
        for (int i = sg.first; i < sg.second; ++i) { lo = std::min(lo, need[i].lo); hi = std::max(hi, need[i].hi); }
        const int s0 = lo / 8 * 8;
        // within a tile, order rows by (j, k): lanes of a warp then share j and read consecutive k (no bank conflicts)
        std::stable_sort(need.begin() + sg.first, need.begin() + sg.second,
                         [](const NeedPair& a, const NeedPair& b) { return std::tie(a.j, a.k) < std::tie(b.j, b.k); });
        tiles.push_back({sg.first, sg.second, s0, round_w(hi + 1 - s0)});
    }
    if (tiles.empty()) tiles.push_back({0, 0, 0, 16});
    // row groups: consecutive tiles while TMEM (two accumulator buffers + two A stages) and the 3 output units allow
    std::vector<std::pair<int, int>> groups;
    for (int t = 0; t < (int)tiles.size();) {
        int e = t, dcols = 0, units = 0;
        while (e < (int)tiles.size() && e - t < opts.group_cap) {
            const int nd = dcols + 2 * tiles[e].W, nu = units + tiles[e].W / 16, nt = e - t + 1;
            if (nu > kMaxUnits || kDBuf * ((nd + 31) / 32 * 32) + 2 * 2 * kKC * nt > 512) break;
            dcols = nd; units = nu; ++e;
        }
        if (e == t) return "contract_tc: tile does not fit tensor memory";
        groups.push_back({t, e});
        t = e;
    }
    if ((int)groups.size() > kMaxGroups) return "contract_tc: more than 4 row groups";
    pl.ngroups = (int)groups.size();

    Params& P = pl.base;
    P = Params{};
    P.ng = ng; P.nh = nh; P.hsep = hsep;
    const int grows = (ng + 7) / 8 * 8;
    P.h_row0 = grows;
    P.slot_bytes = (grows + (hsep ? (nh + 7) / 8 * 8 : 0)) * 128;
    const bool sh = hsep && !sing_g;                        // singles from the h rows
    const int srows = sh ? (nh + 7) / 8 * 8 : grows;       // rows of the singles region of a slot
    P.s_off = sh ? grows * 128 : 0;
    P.s_chunks = srows * 8;
    if (P.s_chunks > 256 * kBloItems) return "contract_tc: more than 64 rows of singles";
    int max_b = 0, max_units = 0;
    rows.assign(tiles.size() * 128, make_short2(-1, -1));
    gidx.assign(std::max(n_out, 1), 0);
    int unit_base = 0;
    for (int gi = 0; gi < pl.ngroups; ++gi) {
        GroupDesc& D = P.grp[gi];
        D = GroupDesc{};
        const int t0 = groups[gi].first, nt = groups[gi].second - t0;
        D.tile0 = t0; D.ntiles = nt; D.unit_base = unit_base;
        // accumulators: [hi*hi | corrections] (2W) of every tile, largest first, so each is aligned to its size
        std::vector<std::pair<int, int>> dl;   // (size, tile)
        for (int t = 0; t < nt; ++t) dl.push_back({2 * tiles[t0 + t].W, t});
        std::stable_sort(dl.begin(), dl.end(), [](auto& a, auto& b) { return a.first > b.first; });
        int col = 0;
        for (auto& x : dl) {
            D.dm_col[x.second] = col;
            col += x.first;
        }
        D.d_cols = (col + 31) / 32 * 32;
        D.a_col0 = kDBuf * D.d_cols;
        D.nA = std::min(kMaxAStages, (512 - D.a_col0) / (2 * kKC * nt));
        // windows of singles; B_lo stages hold a slot's whole singles region
        for (int t = 0; t < nt; ++t) {
            const TileH& T = tiles[t0 + t];
            D.tile_w[t] = T.W;
            D.tile_s0[t] = T.s0;
        }
        D.bstage_bytes = srows * 128;
        max_b = std::max(max_b, D.nA * D.bstage_bytes);
        // output units
        int u = 0;
        for (int t = 0; t < nt; ++t)
            for (int c = 0; c < tiles[t0 + t].W; c += 16) { D.unit_tile[u] = t; D.unit_c[u] = c; ++u; }
        D.nunits = u;
        for (int x = u; x < kMaxUnits; ++x) { D.unit_tile[x] = kMaxTiles; D.unit_c[x] = 0; }
        max_units = std::max(max_units, u);
        // rows and the gather index of every output
        for (int t = 0; t < nt; ++t) {
            const TileH& T = tiles[t0 + t];
            int uf = 0;
            while (D.unit_tile[uf] != t) ++uf;
            for (int i = T.first; i < T.last; ++i) {
                const int r = i - T.first;
                rows[(size_t)(t0 + t) * 128 + r] = make_short2((short)need[i].j, (short)need[i].k);
                for (auto& so : need[i].outs) {
                    const int cc = so.first - T.s0;
                    const int gu = unit_base + uf + cc / 16;
                    gidx[so.second] = (gu * 16 + cc % 16) * 128 + r;
                }
            }
        }
        unit_base += u;
    }
    pl.total_units = unit_base;
    P.total_units = unit_base;
    P.off_b = kRingSlots * P.slot_bytes;
    P.off_acc = P.off_b + max_b;
    P.off_bar = P.off_acc + kMaxUnits * 16 * 128 * 8;
    // + 1024: the kernel aligns the start of its dynamic shared memory to 1024 bytes (128-byte swizzle atoms)
    pl.smem = std::max((size_t)kMinSmem, (size_t)P.off_bar + 64 * 8 + 64) + 1024;
    if (pl.smem > 227 * 1024) return "contract_tc: shared memory plan exceeds 227 KB";

    const long nsl = (ncell + kSlotCells - 1) / kSlotCells;
    const long want = opts.cta_mode == 1 ? std::max(1L, (long)nsm / pl.ngroups) : (opts.cta_mode == 2 ? 2L * nsm : (long)nsm);
    pl.ncta = (int)std::max(1L, std::min(want, nsl));
    pl.cells_cta = (nsl + pl.ncta - 1) / pl.ncta * kSlotCells;
    pl.ncta = (int)((ncell + pl.cells_cta - 1) / pl.cells_cta);
    P.ncell = ncell;
    P.cells_cta = pl.cells_cta;
    return nullptr;
}

static int build_plan(polybin_ctx* ctx, Plan& pl, long ncell, int ng, int nh, int hsep, std::vector<NeedPair> need,
                      int n_out, int sing_g = 0, const PlanOpts& opts = PlanOpts{}, bool quiet = false) {
    int dev = 0, nsm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return fail_cuda(ctx, e, "cudaDeviceGetAttribute", __FILE__, __LINE__);
    std::vector<short2> rows;
    std::vector<int> gidx;
    pl.need = need;
    pl.sing_g = sing_g;
    pl.ncell = ncell;
    const char* msg = layout_plan(pl, ncell, nsm, ng, nh, hsep, std::move(need), n_out, rows, gidx, sing_g, opts);
    if (msg) return quiet ? POLYBIN_EINVAL : fail(ctx, POLYBIN_EINVAL, "%s", msg);
    PB_CUDA_OK(cudaMalloc(&pl.d_rows, sizeof(short2) * rows.size()));
    PB_CUDA_OK(cudaMemcpy(pl.d_rows, rows.data(), sizeof(short2) * rows.size(), cudaMemcpyHostToDevice));
    PB_CUDA_OK(cudaMalloc(&pl.d_gidx, sizeof(int) * gidx.size()));
    PB_CUDA_OK(cudaMemcpy(pl.d_gidx, gidx.data(), sizeof(int) * gidx.size(), cudaMemcpyHostToDevice));
    PB_CUDA_OK(cudaMalloc(&pl.d_partial, sizeof(double) * (size_t)pl.ncta * pl.total_units * 2048));
    pl.base.rows = pl.d_rows;
    pl.base.partial = pl.d_partial;
    return POLYBIN_OK;
}

struct PlanCache {
    std::map<std::tuple<int, int, int, int, long>, Plan*> plans;   // (ng, nh, hsep, kind, ncell)
    double* gram_part = nullptr;                                   // Gram partials (K splits)
    size_t gram_cap = 0;
    ~PlanCache() {
        for (auto& kv : plans) delete kv.second;
        if (gram_part) cudaFree(gram_part);
    }
};

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, []() {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    });
    return fn;
}

// 2D map over `rows` maps of ncell floats (map-major): box = 32 cells x all maps, 128-byte swizzle.
static int make_map(polybin_ctx* ctx, CUtensorMap* m, const float* base, int rows, long ncell) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return fail(ctx, POLYBIN_ECUDA, "contract_tc: cuTensorMapEncodeTiled is not available");
    if (reinterpret_cast<uintptr_t>(base) % 16) return fail(ctx, POLYBIN_EINVAL, "contract_tc: maps must be 16-byte aligned");
    const cuuint64_t dims[2] = {(cuuint64_t)ncell, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)ncell * sizeof(float)};
    const cuuint32_t box[2] = {(cuuint32_t)kSlotCells, (cuuint32_t)rows};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(ctx, POLYBIN_ECUDA, "contract_tc: cuTensorMapEncodeTiled failed (%d)", (int)r);
    return POLYBIN_OK;
}

// 2D map over a row-major float32 matrix [height][width] (row stride width floats), box = box_w x box_h,
// 128-byte swizzle (box_w = 32 floats), out-of-range elements read as zero.
static int make_map2(polybin_ctx* ctx, CUtensorMap* m, const float* base, long width, long height, int box_w, int box_h) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return fail(ctx, POLYBIN_ECUDA, "gram: cuTensorMapEncodeTiled is not available");
    if (reinterpret_cast<uintptr_t>(base) % 16 || (width * (long)sizeof(float)) % 16)
        return fail(ctx, POLYBIN_EINVAL, "gram: rows must be 16-byte aligned");
    const cuuint64_t dims[2] = {(cuuint64_t)width, (cuuint64_t)height};
    const cuuint64_t strides[1] = {(cuuint64_t)width * sizeof(float)};
    const cuuint32_t box[2] = {(cuuint32_t)box_w, (cuuint32_t)box_h};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(ctx, POLYBIN_ECUDA, "gram: cuTensorMapEncodeTiled failed (%d)", (int)r);
    return POLYBIN_OK;
}

static int launch(polybin_ctx* ctx, Plan& pl, const float* g, const float* h, double* d_out) {
    CUtensorMap mg, mh;
    int rc = make_map(ctx, &mg, g, pl.ng, pl.base.ncell);
    if (rc) return rc;
    if (pl.hsep) {
        if ((rc = make_map(ctx, &mh, h, pl.nh, pl.base.ncell))) return rc;
    } else {
        mh = mg;
    }
    if ((rc = ensure_err_flag(ctx))) return rc;
    cudaError_t e = cudaMemsetAsync(ctx->d_err, 0, sizeof(int), ctx->stream);
    if (e != cudaSuccess) return fail_cuda(ctx, e, "cudaMemsetAsync", __FILE__, __LINE__);
    e = cudaFuncSetAttribute((const void*)k_contract_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl.smem);
    if (e != cudaSuccess) return fail_cuda(ctx, e, "cudaFuncSetAttribute(k_contract_tc)", __FILE__, __LINE__);
    {
        // the setmaxnreg split assumes exactly kRegsLaunch registers a thread at launch (a smaller allocation would
        // leave the producers' increase waiting for registers that do not exist)
        cudaFuncAttributes fa{};
        e = cudaFuncGetAttributes(&fa, (const void*)k_contract_tc);
        if (e != cudaSuccess) return fail_cuda(ctx, e, "cudaFuncGetAttributes(k_contract_tc)", __FILE__, __LINE__);
        if (fa.numRegs != kRegsLaunch)
            return fail(ctx, POLYBIN_ECUDA, "contract_tc: kernel built with %d registers a thread, %d expected", fa.numRegs,
                        kRegsLaunch);
    }
    Params P = pl.base;
    P.err = ctx->d_err;
    {
        StageTimer timer(ctx, kStageContract);
        k_contract_tc<<<dim3(pl.ncta, pl.ngroups, 1), kThreads, pl.smem, ctx->stream>>>(mg, mh, P);
        ctx->launches += 1;
        e = cudaGetLastError();
        if (e != cudaSuccess) return fail_cuda(ctx, e, "k_contract_tc", __FILE__, __LINE__);
        k_reduce_gather<<<(pl.n_out + 255) / 256, 256, 0, ctx->stream>>>(pl.d_partial, pl.ncta,
                                                                          (long)pl.total_units * 2048, pl.d_gidx,
                                                                          pl.n_out, d_out);
        ctx->launches += 1;
        e = cudaGetLastError();
        if (e != cudaSuccess) return fail_cuda(ctx, e, "k_reduce_gather", __FILE__, __LINE__);
    }
    if (ctx->capturing) return POLYBIN_OK;   // the caller reads the error flags after the graph has run
    return read_err_flags(ctx, "contract_tc");
}

static PlanCache* cache_of(polybin_ctx* ctx) {
    if (!ctx->tc) ctx->tc = new PlanCache();
    return static_cast<PlanCache*>(ctx->tc);
}

// Autotuner.  On the first launch of a plan outside stream capture (unless POLYBIN_AUTOTUNE=0), every distinct valid
// candidate of the option grid {tile cost 8, 24} x {3 or 1 tiles a group} x {cell splits 0, 1, 2} runs on the
// caller's own inputs, timed with CUDA events on the context stream (one launch to warm up, two timed); the fastest
// replaces the plan in the cache.  Candidates differ only in how cells and rows are split, so their results agree to
// FP32 rounding of the partial sums; after tuning every call takes the chosen plan.
static int tune_plan(polybin_ctx* ctx, Plan** pl_io, const float* g, const float* h, double* d_out) {
    Plan* pl = *pl_io;
    if (pl->tuned) return POLYBIN_OK;
    if (ctx->capturing) {   // a captured graph keeps this plan's buffers: it must never be replaced
        pl->tuned = true;
        return POLYBIN_OK;
    }
    const char* env = std::getenv("POLYBIN_AUTOTUNE");
    if (env && env[0] == '0') { pl->tuned = true; return POLYBIN_OK; }
    PlanCache* pc = cache_of(ctx);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    PB_CUDA_OK(cudaEventCreate(&e0));
    PB_CUDA_OK(cudaEventCreate(&e1));
    auto time_plan = [&](Plan& c, float* ms) -> int {
        int rc;
        if ((rc = launch(ctx, c, g, h, d_out))) return rc;
        PB_CUDA_OK(cudaEventRecord(e0, ctx->stream));
        for (int i = 0; i < 2; ++i)
            if ((rc = launch(ctx, c, g, h, d_out))) return rc;
        PB_CUDA_OK(cudaEventRecord(e1, ctx->stream));
        PB_CUDA_OK(cudaEventSynchronize(e1));
        PB_CUDA_OK(cudaEventElapsedTime(ms, e0, e1));
        *ms *= 0.5f;
        return POLYBIN_OK;
    };
    float best_ms = 0.f;
    int rc = time_plan(*pl, &best_ms);
    Plan* best = pl;
    int tried = 1;
    std::vector<Plan*> others;
    auto sig = [](const Plan& c) {   // (tiles, groups, ncta, cells a CTA, units): equal signatures, equal launches
        int nt = 0;
        for (int i = 0; i < c.ngroups; ++i) nt += c.base.grp[i].ntiles;
        return std::make_tuple(nt, c.ngroups, c.ncta, c.cells_cta, c.total_units);
    };
    std::set<std::tuple<int, int, int, long, int>> seen;
    seen.insert(sig(*pl));
    const int costs[2] = {8, 24}, caps[2] = {kMaxTiles, 1};
    for (int ci = 0; ci < 2 && !rc; ++ci)
        for (int gi = 0; gi < 2 && !rc; ++gi)
            for (int mode = 0; mode < 3 && !rc; ++mode) {
                PlanOpts o;
                o.tile_cost = costs[ci];
                o.group_cap = caps[gi];
                o.cta_mode = mode;
                Plan* c = new Plan();
                if (build_plan(ctx, *c, pl->ncell, pl->ng, pl->nh, pl->hsep, pl->need, pl->n_out, pl->sing_g, o, true)) {
                    delete c;
                    continue;
                }
                if (!seen.insert(sig(*c)).second) { delete c; continue; }
                float ms = 0.f;
                rc = time_plan(*c, &ms);
                ++tried;
                others.push_back(c);
                if (!rc && ms < best_ms) { best_ms = ms; best = c; }
            }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    // keep the winner in the cache slot of the original plan
    for (auto& kv : pc->plans)
        if (kv.second == pl) kv.second = best;
    if (best != pl) delete pl;
    for (Plan* c : others)
        if (c != best) delete c;
    best->tuned = true;
    best->tuned_ms = best_ms;
    best->tuned_of = tried;
    *pl_io = best;
    return rc;
}

static int launch_tuned(polybin_ctx* ctx, Plan* pl, const float* g, const float* h, double* d_out) {
    int rc;
    if ((rc = tune_plan(ctx, &pl, g, h, d_out))) return rc;
    return launch(ctx, *pl, g, h, d_out);
}

// Plan of all pairs (j <= k) of ng maps against the nh singles [0, nh), output M[(j, k)][i] pair-major.
static int full_plan(polybin_ctx* ctx, long ncell, int ng, int nh, int hsep, Plan** out) {
    PlanCache* pc = cache_of(ctx);
    auto key = std::make_tuple(ng, nh, hsep, 0, ncell);
    auto it = pc->plans.find(key);
    if (it != pc->plans.end()) { *out = it->second; return POLYBIN_OK; }
    std::vector<NeedPair> need;
    int p = 0;
    for (int j = 0; j < ng; ++j)
        for (int k = j; k < ng; ++k, ++p) {
            NeedPair np{j, k, 0, nh - 1, {}};
            for (int i = 0; i < nh; ++i) np.outs.push_back({i, p * nh + i});
            need.push_back(std::move(np));
        }
    Plan* pl = new Plan();
    int rc = build_plan(ctx, *pl, ncell, ng, nh, hsep, std::move(need), p * nh);
    if (rc) { delete pl; return rc; }
    pc->plans[key] = pl;
    *out = pl;
    return POLYBIN_OK;
}

// Plan of the closed triplets of the context on the contraction grid: triplet a <= b <= c from pair (b, c) and
// single a, output S' in triplet order.
static int triplet_plan(polybin_ctx* ctx, Plan** out) {
    PlanCache* pc = cache_of(ctx);
    const int nb = ctx->nb;
    auto key = std::make_tuple(nb, nb, 0, 1, ctx->cg.ncell);
    auto it = pc->plans.find(key);
    if (it != pc->plans.end()) { *out = it->second; return POLYBIN_OK; }
    std::map<std::pair<int, int>, NeedPair> m;
    const int nt = (int)ctx->Nabc.size();
    for (int t = 0; t < nt; ++t) {
        const int a = ctx->trip[3 * t], b = ctx->trip[3 * t + 1], c = ctx->trip[3 * t + 2];
        auto f = m.find({b, c});
        if (f == m.end()) f = m.emplace(std::make_pair(b, c), NeedPair{b, c, a, a, {}}).first;
        f->second.lo = std::min(f->second.lo, a);
        f->second.hi = std::max(f->second.hi, a);
        f->second.outs.push_back({a, t});
    }
    std::vector<NeedPair> need;
    for (auto& kv : m) need.push_back(std::move(kv.second));
    Plan* pl = new Plan();
    int rc = build_plan(ctx, *pl, ctx->cg.ncell, nb, nb, 0, std::move(need), nt);
    if (rc) { delete pl; return rc; }
    pc->plans[key] = pl;
    *out = pl;
    return POLYBIN_OK;
}

// Plan of the closed triplets for a multipole ell > 0 (Sec. 4.1, eq. ideal-bk: L_ell on the third bin): triplet
// a <= b <= c from the pair (g_b, g_{c,ell}) -- g_b a row of the g maps, g_{c,ell} a row of the h maps in the
// same slot -- and the single g_a, output S^ell' in triplet order.  Same pairs and windows as the ell = 0 plan.
static int ell_plan(polybin_ctx* ctx, Plan** out) {
    PlanCache* pc = cache_of(ctx);
    const int nb = ctx->nb;
    auto key = std::make_tuple(nb, nb, 1, 2, ctx->cg.ncell);
    auto it = pc->plans.find(key);
    if (it != pc->plans.end()) { *out = it->second; return POLYBIN_OK; }
    const int h0 = (nb + 7) / 8 * 8;
    std::map<std::pair<int, int>, NeedPair> m;
    const int nt = (int)ctx->Nabc.size();
    for (int t = 0; t < nt; ++t) {
        const int a = ctx->trip[3 * t], b = ctx->trip[3 * t + 1], c = ctx->trip[3 * t + 2];
        auto f = m.find({b, c});
        if (f == m.end()) f = m.emplace(std::make_pair(b, c), NeedPair{b, h0 + c, a, a, {}}).first;
        f->second.lo = std::min(f->second.lo, a);
        f->second.hi = std::max(f->second.hi, a);
        f->second.outs.push_back({a, t});
    }
    std::vector<NeedPair> need;
    for (auto& kv : m) need.push_back(std::move(kv.second));
    Plan* pl = new Plan();
    int rc = build_plan(ctx, *pl, ctx->cg.ncell, nb, nb, 1, std::move(need), nt, 1);
    if (rc) { delete pl; return rc; }
    pc->plans[key] = pl;
    *out = pl;
    return POLYBIN_OK;
}

}  // namespace tc

bool split_tc_available() { return true; }

// Runs k_tf32_selfcheck once per device (the first split-TF32 context on it); POLYBIN_ETOL if the tensor core does
// not read FP32 operands as the split scheme assumes.
int tf32_selfcheck(polybin_ctx* ctx) {
    static std::mutex mu;
    static int state[256] = {};   // 0 unchecked, 1 ok, -1 failed
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail_cuda(ctx, e, "cudaGetDevice", __FILE__, __LINE__);
    if (dev < 0 || dev >= 256) return POLYBIN_OK;
    std::lock_guard<std::mutex> lock(mu);
    if (state[dev] == 0) {
        uint32_t* d = nullptr;
        uint32_t h[3] = {0u, 0u, 1u};
        e = cudaMalloc(&d, sizeof(h));
        if (e == cudaSuccess) e = cudaMemsetAsync(d, 0, sizeof(h), ctx->stream);
        if (e == cudaSuccess) {
            tc::k_tf32_selfcheck<<<1, 128, 0, ctx->stream>>>(d);
            ctx->launches += 1;
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaMemcpyAsync(h, d, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        if (d) cudaFree(d);
        if (e != cudaSuccess) return fail_cuda(ctx, e, "tf32 self-check", __FILE__, __LINE__);
        float d00, d10;
        std::memcpy(&d00, &h[0], 4);
        std::memcpy(&d10, &h[1], 4);
        state[dev] = (h[2] == 0u && d00 == 1.0f && d10 == 1.0f + 0x1p-10f) ? 1 : -1;
        if (state[dev] < 0)
            return fail(ctx, POLYBIN_ETOL, "tf32 self-check: D00 = %.9g, D10 = %.9g (expected 1 and 1 + 2^-10): the tensor "
                        "core does not read FP32 operands as TF32 by truncation", (double)d00, (double)d10);
    }
    if (state[dev] < 0)
        return fail(ctx, POLYBIN_ETOL, "tf32 self-check failed on this device: split-TF32 mode unavailable");
    return POLYBIN_OK;
}

void destroy_tc(polybin_ctx* ctx) {
    delete static_cast<tc::PlanCache*>(ctx->tc);
    ctx->tc = nullptr;
}

int ensure_err_flag(polybin_ctx* ctx) {
    if (ctx->d_err) return POLYBIN_OK;
    cudaError_t e = cudaMalloc(&ctx->d_err, kErrFlags * sizeof(int));
    if (e != cudaSuccess) return fail_cuda(ctx, e, "cudaMalloc err flag", __FILE__, __LINE__);
    e = cudaMemset(ctx->d_err, 0, kErrFlags * sizeof(int));
    if (e != cudaSuccess) return fail_cuda(ctx, e, "cudaMemset err flag", __FILE__, __LINE__);
    return POLYBIN_OK;
}

// Reads both error flags after the work queued on the stream (synchronising it).  The staging flag is raised by the
// transform passes that run before the contraction on the same stream and is cleared once reported.
int read_err_flags(polybin_ctx* ctx, const char* what) {
    int herr[kErrFlags] = {0, 0};
    cudaError_t e = cudaMemcpyAsync(herr, ctx->d_err, sizeof(herr), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return fail_cuda(ctx, e, "error flags", __FILE__, __LINE__);
    if (herr[kErrStaging]) {
        e = cudaMemset(ctx->d_err + kErrStaging, 0, sizeof(int));
        if (e != cudaSuccess) return fail_cuda(ctx, e, "cudaMemset err flag", __FILE__, __LINE__);
        return fail(ctx, POLYBIN_ETIMEOUT, "%s: a bulk staging copy of a transform pass did not complete", what);
    }
    if (herr[kErrPipeline]) return fail(ctx, POLYBIN_ETIMEOUT, "%s: a pipeline wait timed out", what);
    return POLYBIN_OK;
}

// Shapes the tensor-core kernel takes: <= 512 pairs, <= 32 singles, cells a multiple of 4, 16-byte aligned maps.
bool tc_shape_ok(long ncell, const float* g, int ng, const float* h, int nh) {
    if (ng < 1 || ng * (ng + 1) / 2 > 512 || nh < 1 || nh > 32) return false;
    if (ncell % 4 || ncell > 0x7fffffffL) return false;
    if (reinterpret_cast<uintptr_t>(g) % 16 || (h && reinterpret_cast<uintptr_t>(h) % 16)) return false;
    return true;
}

// M[(j <= k)][i] (pair-major, device) of ng maps g against nh singles h (h == nullptr: h = g), over ncell cells.
int run_contract_tc(polybin_ctx* ctx, const float* g, int ng, const float* h, int nh, double* d_out, long ncell) {
    const int hsep = (h && h != g) ? 1 : 0;
    if (!hsep) nh = ng;
    tc::Plan* pl = nullptr;
    int rc = tc::full_plan(ctx, ncell, ng, nh, hsep, &pl);
    if (rc) return rc;
    return tc::launch_tuned(ctx, pl, g, hsep ? h : g, d_out);
}

// Builds the closed-triplet plan ahead of time (before any stream capture).
int prepare_triplet_tc(polybin_ctx* ctx) {
    tc::Plan* pl = nullptr;
    return tc::triplet_plan(ctx, &pl);
}

// S^ell'_abc = sum g_a g_b g_{c,ell} of every closed triplet (device, triplet order) from the shell maps g and the
// Legendre-weighted maps gl on the contraction grid.
int run_triplet_sums_ell_tc(polybin_ctx* ctx, const float* g, const float* gl, double* d_S) {
    tc::Plan* pl = nullptr;
    int rc = tc::ell_plan(ctx, &pl);
    if (rc) return rc;
    return tc::launch_tuned(ctx, pl, g, gl, d_S);
}

// out[i][j] += scale sum_k A[i][k] B[j][k] for float32 rows A [nA][K], B [nB][K] (K a multiple of 4, 16-byte aligned
// rows) on the tensor cores (3-term split TF32, FP64 sums across K splits in a fixed order).
int run_gram_tc(polybin_ctx* ctx, const float* A, int nA, const float* B, int nB, long K, double scale, double* d_out) {
    using namespace tc::gram;
    if (nA < 1 || nB < 1 || K < 1) return POLYBIN_OK;
    tc::PlanCache* pc = tc::cache_of(ctx);
    CUtensorMap mA, mB;
    int rc = tc::make_map2(ctx, &mA, A, K, nA, kKC, kBM);
    if (rc) return rc;
    if ((rc = tc::make_map2(ctx, &mB, B, K, nB, kKC, kBN))) return rc;
    const int nI = (nA + kBM - 1) / kBM, nJ = (nB + kBN - 1) / kBN;
    int dev = 0, nsm = 0;
    PB_CUDA_OK(cudaGetDevice(&dev));
    PB_CUDA_OK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const long kst = (K + kKC - 1) / kKC;
    int nsplit = (int)std::max(1L, std::min(kst, (long)((2 * nsm + nI * nJ - 1) / (nI * nJ))));
    const long k_cta = (kst + nsplit - 1) / nsplit * kKC;
    nsplit = (int)((K + k_cta - 1) / k_cta);
    const long ldp = (long)nJ * kBN, split_stride = (long)nI * kBM * ldp;
    const size_t need = (size_t)nsplit * split_stride;
    if (need > pc->gram_cap) {
        if (pc->gram_part) cudaFree(pc->gram_part);
        pc->gram_part = nullptr;
        pc->gram_cap = 0;
        PB_CUDA_OK(cudaMalloc(&pc->gram_part, sizeof(double) * need));
        pc->gram_cap = need;
    }
    if ((rc = ensure_err_flag(ctx))) return rc;
    PB_CUDA_OK(cudaMemsetAsync(ctx->d_err, 0, sizeof(int), ctx->stream));
    PB_CUDA_OK(cudaFuncSetAttribute((const void*)k_gram_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem));
    {
        cudaFuncAttributes fa{};
        PB_CUDA_OK(cudaFuncGetAttributes(&fa, (const void*)k_gram_tc));
        if (fa.numRegs * kThreads > 65536)
            return fail(ctx, POLYBIN_ECUDA, "gram: kernel built with %d registers a thread", fa.numRegs);
    }
    GP P;
    P.k_cta = k_cta; P.K = K; P.nA = nA; P.nB = nB; P.nsplit = nsplit;
    P.part = pc->gram_part; P.ldp = ldp; P.split_stride = split_stride; P.err = ctx->d_err;
    k_gram_tc<<<dim3(nJ, nI, nsplit), kThreads, kSmem, ctx->stream>>>(mA, mB, P);
    ctx->launches += 1;
    PB_CUDA_OK(cudaGetLastError());
    const long nout = (long)nA * nB;
    k_gram_reduce<<<(unsigned)((nout + 255) / 256), 256, 0, ctx->stream>>>(pc->gram_part, nsplit, split_stride, ldp, nA, nB,
                                                                          scale, d_out);
    ctx->launches += 1;
    PB_CUDA_OK(cudaGetLastError());
    return read_err_flags(ctx, "gram");
}

// S'_abc of every closed triplet (device, triplet order) from the shell maps g on the contraction grid.
int run_triplet_sums_tc(polybin_ctx* ctx, const float* g, double* d_S) {
    tc::Plan* pl = nullptr;
    int rc = tc::triplet_plan(ctx, &pl);
    if (rc) return rc;
    return tc::launch_tuned(ctx, pl, g, g, d_S);
}

}  // namespace pb

extern "C" int polybin_selftest_wait(polybin_ctx* ctx, int* timed_out) {
    if (!ctx || !timed_out) return pb::fail(ctx, POLYBIN_EINVAL, "polybin_selftest_wait: NULL argument");
    int rc = pb::ensure_err_flag(ctx);
    if (rc) return rc;
    PB_CUDA_OK(cudaMemsetAsync(ctx->d_err, 0, pb::kErrFlags * sizeof(int), ctx->stream));
    pb::tc::k_wait_selftest<<<1, 32, 0, ctx->stream>>>(ctx->d_err + pb::kErrPipeline, 1u << 14);
    ctx->launches++;
    PB_CUDA_OK(cudaGetLastError());
    if ((rc = pb::run_bulk_wait_selftest(ctx, 1u << 14))) return rc;
    int h[pb::kErrFlags] = {0, 0};
    PB_CUDA_OK(cudaMemcpyAsync(h, ctx->d_err, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream));
    PB_CUDA_OK(cudaStreamSynchronize(ctx->stream));
    PB_CUDA_OK(cudaMemsetAsync(ctx->d_err, 0, pb::kErrFlags * sizeof(int), ctx->stream));
    *timed_out = (h[pb::kErrPipeline] && h[pb::kErrStaging]) ? 1 : 0;
    return POLYBIN_OK;
}

// The closed-triplet plan of the context's tensor-core contraction (ell = 0) and what the autotuner chose.
extern "C" int polybin_contract_plan_info(polybin_ctx* ctx, int info[6], float* ms) {
    if (!ctx || !info) return pb::fail(ctx, POLYBIN_EINVAL, "polybin_contract_plan_info: NULL argument");
    for (int i = 0; i < 6; ++i) info[i] = -1;
    if (ms) *ms = 0.f;
    if (!ctx->tc) return POLYBIN_OK;
    pb::tc::PlanCache* pc = static_cast<pb::tc::PlanCache*>(ctx->tc);
    auto it = pc->plans.find(std::make_tuple(ctx->nb, ctx->nb, 0, 1, ctx->cg.ncell));
    if (it == pc->plans.end()) return POLYBIN_OK;
    const pb::tc::Plan& p = *it->second;
    info[0] = p.opts.tile_cost;
    info[1] = p.opts.group_cap;
    info[2] = p.opts.cta_mode;
    info[3] = p.ngroups;
    info[4] = p.ncta;
    info[5] = p.tuned ? p.tuned_of : 0;
    if (ms) *ms = p.tuned_ms;
    return POLYBIN_OK;
}
