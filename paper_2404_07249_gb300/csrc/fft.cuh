// Mixed-radix (2, 3, 4, 5, 8) Stockham FFT staged in shared memory, and the pass kernels of the
// pruned 3D real transforms used by the estimators:
//   forward  (R2C):  z-pass on pairs of real lines -> y-pass -> x-pass, keeping only the box of wave
//                    numbers that any k-bin can reach (|n_i| <= m);
//   inverse  (C2R):  x-pass that applies the shell filter Theta_b on load -> y-pass -> z-pass on pairs
//                    of Hermitian half-lines, per bin b over that bin's own bounding box.
// A line of length n lives in shared memory as element (l, e) at l + e * ES, so that consecutive
// threads touch consecutive lines (conflict-free) in every radix pass.
#pragma once
#include <type_traits>

#include "common.cuh"
#include "ylm.cuh"

namespace pb {

constexpr int kMaxPasses = 12;
constexpr int kMaxItems = 64;

struct FftPlan {
    int n;
    int nr;
    int radix[kMaxPasses];
};

// Factor n into radices 8, 4, 2, 3, 5 (largest power-of-two radices first).  False if n has another
// prime factor or is too long for shared-memory staging.
inline bool make_plan(int n, FftPlan& p) {
    p.n = n;
    p.nr = 0;
    if (n < 2 || n > 1024) return false;
    int m = n;
    while (m % 8 == 0) { p.radix[p.nr++] = 8; m /= 8; }
    while (m % 4 == 0) { p.radix[p.nr++] = 4; m /= 4; }
    while (m % 2 == 0) { p.radix[p.nr++] = 2; m /= 2; }
    while (m % 3 == 0) { p.radix[p.nr++] = 3; m /= 3; }
    while (m % 5 == 0) { p.radix[p.nr++] = 5; m /= 5; }
    return m == 1 && p.nr <= kMaxPasses;
}

// In-register DFT of length R (R in {2,3,4,5,8}); DIR = -1 forward (e^{-2 pi i}), +1 inverse.
template <typename T, int DIR>
__device__ __forceinline__ void dft4(C<T>& a0, C<T>& a1, C<T>& a2, C<T>& a3) {
    C<T> t0 = add<T>(a0, a2), t1 = sub<T>(a0, a2), t2 = add<T>(a1, a3), t3 = sub<T>(a1, a3);
    // w = e^{DIR 2 pi i / 4} = DIR * i
    C<T> wt3 = muli<T>(t3, DIR);
    a0 = add<T>(t0, t2);
    a2 = sub<T>(t0, t2);
    a1 = add<T>(t1, wt3);
    a3 = sub<T>(t1, wt3);
}

template <typename T, int DIR>
__device__ __forceinline__ void dft(C<T>* v, int R) {
    const T h = T(0.70710678118654752440);  // sqrt(1/2)
    switch (R) {
        case 2: {
            C<T> a = v[0], b = v[1];
            v[0] = add<T>(a, b);
            v[1] = sub<T>(a, b);
        } break;
        case 4: dft4<T, DIR>(v[0], v[1], v[2], v[3]); break;
        case 8: {
            C<T> e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
            C<T> o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
            dft4<T, DIR>(e0, e1, e2, e3);
            dft4<T, DIR>(o0, o1, o2, o3);
            // o_q *= w8^q, w8 = e^{DIR 2 pi i / 8} = h (1 + DIR i)
            o1 = mk<T>(h * (o1.x - DIR * o1.y), h * (o1.y + DIR * o1.x));
            o2 = muli<T>(o2, DIR);
            o3 = mk<T>(h * (-o3.x - DIR * o3.y), h * (-o3.y + DIR * o3.x));
            v[0] = add<T>(e0, o0); v[4] = sub<T>(e0, o0);
            v[1] = add<T>(e1, o1); v[5] = sub<T>(e1, o1);
            v[2] = add<T>(e2, o2); v[6] = sub<T>(e2, o2);
            v[3] = add<T>(e3, o3); v[7] = sub<T>(e3, o3);
        } break;
        case 3: {
            const T s3 = T(0.86602540378443864676);  // sin(2 pi / 3)
            C<T> s = add<T>(v[1], v[2]), d = sub<T>(v[1], v[2]);
            C<T> t = mk<T>(v[0].x - T(0.5) * s.x, v[0].y - T(0.5) * s.y);
            C<T> id = muli<T>(d, DIR);
            v[0] = add<T>(v[0], s);
            v[1] = mk<T>(t.x + s3 * id.x, t.y + s3 * id.y);
            v[2] = mk<T>(t.x - s3 * id.x, t.y - s3 * id.y);
        } break;
        case 5: {
            const T c1 = T(0.30901699437494742410), c2 = T(-0.80901699437494742410);   // cos(2pi/5), cos(4pi/5)
            const T s1 = T(0.95105651629515357212), s2 = T(0.58778525229247312917);    // sin(2pi/5), sin(4pi/5)
            C<T> a0 = v[0];
            C<T> p1 = add<T>(v[1], v[4]), m1 = sub<T>(v[1], v[4]);
            C<T> p2 = add<T>(v[2], v[3]), m2 = sub<T>(v[2], v[3]);
            C<T> r1 = mk<T>(a0.x + c1 * p1.x + c2 * p2.x, a0.y + c1 * p1.y + c2 * p2.y);
            C<T> r2 = mk<T>(a0.x + c2 * p1.x + c1 * p2.x, a0.y + c2 * p1.y + c1 * p2.y);
            C<T> q1 = muli<T>(mk<T>(s1 * m1.x + s2 * m2.x, s1 * m1.y + s2 * m2.y), DIR);
            C<T> q2 = muli<T>(mk<T>(s2 * m1.x - s1 * m2.x, s2 * m1.y - s1 * m2.y), DIR);
            v[0] = add<T>(a0, add<T>(p1, p2));
            v[1] = add<T>(r1, q1);
            v[4] = sub<T>(r1, q1);
            v[2] = add<T>(r2, q2);
            v[3] = sub<T>(r2, q2);
        } break;
        default: break;
    }
}

// Stockham autosort FFT of L lines (element (l, e) at l + e * ES) using a ping-pong buffer pair.
// tw[m] = e^{-2 pi i m / n}.  Returns the buffer holding the result (natural order).
// Pass with radix R after Ns = product of earlier radices: butterfly j (0 <= j < n/R), k = j mod Ns,
// reads x[j + r n/R] (r < R), multiplies by w^{r k n/(Ns R)}, takes the R-point DFT and writes
// output q to position (j - k) R + k + q Ns.
template <typename T, int DIR>
__device__ C<T>* fft_lines(C<T>* src, C<T>* dst, int L, int ES, const FftPlan& p, const C<T>* __restrict__ tw,
                           int tid, int nthr) {
    const int n = p.n;
    int Ns = 1;
    for (int pass = 0; pass < p.nr; ++pass) {
        const int R = p.radix[pass];
        const int nbf = n / R;
        const int tstride = n / (Ns * R);
        const int total = nbf * L;
        for (int w = tid; w < total; w += nthr) {
            const int l = w % L;
            const int j = w / L;
            const int k = j % Ns;
            C<T> v[8];
#pragma unroll
            for (int r = 0; r < 8; ++r)
                if (r < R) v[r] = src[l + (j + r * nbf) * ES];
            if (Ns > 1) {
#pragma unroll
                for (int r = 1; r < 8; ++r)
                    if (r < R) {
                        C<T> t = tw[r * k * tstride];
                        v[r] = DIR < 0 ? mul<T>(v[r], t) : mulc<T>(v[r], t);
                    }
            }
            dft<T, DIR>(v, R);
            const int base = (j - k) * R + k;
#pragma unroll
            for (int q = 0; q < 8; ++q)
                if (q < R) dst[l + (base + q * Ns) * ES] = v[q];
        }
        __syncthreads();
        C<T>* t = src;
        src = dst;
        dst = t;
        Ns *= R;
    }
    return src;
}


// ------------------------------------------------------------------------------------------------
// Compile-time specialisation for the lengths listed in PB_WITH_NT: radices, strides and line counts are
// constants, so the index arithmetic folds and every radix loop is fully unrolled.  The radix order is that of
// make_plan (8s, then 4, 2, 3s, 5s).
// Shared-memory budgets of the staged passes (ping-pong buffers of one CTA): they set the lines a z-pass CTA and
// the columns a strided-pass CTA transform, and with them how many CTAs an SM holds.
#ifndef PB_LINES_SMEM
#define PB_LINES_SMEM (48 * 1024)
#endif
#ifndef PB_COLS_SMEM
#define PB_COLS_SMEM (64 * 1024)
#endif
template <typename T> __host__ __device__ constexpr int lines_per_cta_of(int n) {
    int lp = 16;
    while (lp > 1 && 2 * (long)n * (lp + 1) * (long)sizeof(C<T>) > PB_LINES_SMEM) lp >>= 1;
    return lp;
}
template <typename T> __host__ __device__ constexpr int cols_per_cta_of(int n) {
    int tk = 16;
    while (tk > 1 && 2 * (long)n * tk * (long)sizeof(C<T>) > PB_COLS_SMEM) tk >>= 1;
    return tk;
}
__host__ __device__ constexpr int ct_next_radix(int m) {
    return m % 8 == 0 ? 8 : (m % 4 == 0 ? 4 : (m % 2 == 0 ? 2 : (m % 3 == 0 ? 3 : (m % 5 == 0 ? 5 : 1))));
}
__host__ __device__ constexpr int ct_radix(int n, int pass) {
    int m = n;
    for (int p = 0; p < pass; ++p) m /= ct_next_radix(m);
    return m <= 1 ? 1 : ct_next_radix(m);
}
__host__ __device__ constexpr int ct_passes(int n) {
    int c = 0;
    while (ct_radix(n, c) > 1) ++c;
    return c;
}

template <typename T, int DIR, int N, int L, int ES, int NTHR, int PASS, int NS>
__device__ __forceinline__ C<T>* fft_ct_pass(C<T>* src, C<T>* dst, const C<T>* __restrict__ tw, int tid) {
    if constexpr (PASS == ct_passes(N)) {
        return src;
    } else {
        constexpr int R = ct_radix(N, PASS);
        constexpr int NBF = N / R;
        constexpr int TSTR = N / (NS * R);
        constexpr int TOTAL = NBF * L;
#pragma unroll 2
        for (int w = tid; w < TOTAL; w += NTHR) {
            const int l = w % L;
            const int j = w / L;
            const int k = j % NS;
            C<T> v[8];
#pragma unroll
            for (int r = 0; r < R; ++r) v[r] = src[l + (j + r * NBF) * ES];
            if constexpr (NS > 1) {
#pragma unroll
                for (int r = 1; r < R; ++r) {
                    const C<T> t = tw[r * k * TSTR];
                    v[r] = DIR < 0 ? mul<T>(v[r], t) : mulc<T>(v[r], t);
                }
            }
            dft<T, DIR>(v, R);
            const int base = (j - k) * R + k;
#pragma unroll
            for (int q = 0; q < R; ++q) dst[l + (base + q * NS) * ES] = v[q];
        }
        __syncthreads();
        return fft_ct_pass<T, DIR, N, L, ES, NTHR, PASS + 1, NS * R>(dst, src, tw, tid);
    }
}

// Dispatch: compile-time version when NT > 0, run-time plan otherwise.
template <typename T, int DIR, int NT, int LT, int ET>
__device__ __forceinline__ C<T>* fft_any(C<T>* src, C<T>* dst, int L, int ES, const FftPlan& p,
                                         const C<T>* __restrict__ tw, int tid, int nthr) {
    if constexpr (NT > 0) {
        return fft_ct_pass<T, DIR, NT, LT, ET, 256, 0, 1>(src, dst, tw, tid);
    } else {
        return fft_lines<T, DIR>(src, dst, L, ES, p, tw, tid, nthr);
    }
}

// Twiddles e^{-2 pi i m / n} staged into shared memory (after a __syncthreads they are visible to the CTA).
template <typename T>
__device__ __forceinline__ void stage_twiddles(C<T>* dst, const C<T>* __restrict__ tw, int n, int tid, int nthr) {
    for (int i = tid; i < n; i += nthr) dst[i] = tw[i];
}

// One-shot bulk copy global -> shared through the TMA engine (cp.async.bulk: both addresses 16-byte aligned, size a
// multiple of 16), completing on an mbarrier with the byte count; and the bounded wait on that barrier.
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void bulk_bar_init(uint64_t* bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n\tfence.mbarrier_init.release.cluster;" ::"r"(smem_addr(bar))
                 : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "fence.proxy.async.shared::cta;\n\t"
        "mbarrier.arrive.expect_tx.shared::cta.b64 _, [%2], %3;\n\t"
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %3, [%2];" ::"r"(smem_addr(dst)),
        "l"(src), "r"(smem_addr(bar)), "r"(bytes)
        : "memory");
}
// Waits for phase `parity` of the barrier; false after `limit` polls (the copy never landed).
__device__ __forceinline__ bool bulk_wait(uint64_t* bar, uint32_t parity, unsigned limit) {
    for (unsigned it = 0; it < limit; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(smem_addr(bar)), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}
constexpr unsigned kBulkSpinLimit = 1u << 22;
// Self-test of the staging wait: a barrier armed for 16 bytes that no copy delivers (none is issued); the bounded
// wait gives up and raises the flag.
static __global__ void k_bulk_wait_selftest(int* err, unsigned limit) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        bulk_bar_init(&bar);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], 16;" ::"r"(smem_addr(&bar)) : "memory");
        if (!bulk_wait(&bar, 0u, limit)) atomicExch(err, 1);
    }
}

// ------------------------------------------------------------------------------------------------
// z-pass, forward: pairs of real lines (lines 2p, 2p+1 of the flattened (x, y) index) packed as one
// complex line, transformed, then split into the two Hermitian half-spectra; only kz < kout is stored.
// Optional pointwise multipliers m1, m2 (same layout as the input) are applied on load.
template <typename T, typename TIN, typename TM, int NT = 0>
__global__ void __launch_bounds__(256) k_fwd_z(const TIN* __restrict__ in, const TM* __restrict__ m1,
                                               const TM* __restrict__ m2, C<T>* __restrict__ out, long nlines,
                                               int kout, FftPlan plan, const C<T>* __restrict__ twg, int LPrt) {
    extern __shared__ unsigned char smem_raw[];
    constexpr int LT = NT > 0 ? lines_per_cta_of<T>(NT) : 0;
    const int n = NT > 0 ? NT : plan.n;
    const int LP = NT > 0 ? LT : LPrt;
    const int ES = LP + 1;
    C<T>* b0 = reinterpret_cast<C<T>*>(smem_raw);
    C<T>* b1 = b0 + (size_t)n * ES;
    C<T>* tw = b1 + (size_t)n * ES;
    const long line0 = (long)blockIdx.x * 2 * LP;
    const int tid = threadIdx.x, nthr = blockDim.x;
    stage_twiddles<T>(tw, twg, n, tid, nthr);
    T* bs = reinterpret_cast<T*>(b0);
    if constexpr (NT > 0) {
        // compile-time trip count (256 threads): every load of the CTA's lines is issued before the first store, so
        // the global latency is paid once rather than once per element
        constexpr int TOT = 2 * LT * NT;
        constexpr int IT = (TOT + 255) / 256;
        T vals[IT];
#pragma unroll
        for (int q = 0; q < IT; ++q) {
            const int idx = tid + 256 * q;
            const int r = idx / NT, e = idx - r * NT;
            const long gl = line0 + r;
            T v = T(0);
            if (idx < TOT && gl < nlines) {
                const long gi = gl * NT + e;
                v = T(in[gi]);
                if (m1) v *= T(m1[gi]);
                if (m2) v *= T(m2[gi]);
            }
            vals[q] = v;
        }
#pragma unroll
        for (int q = 0; q < IT; ++q) {
            const int idx = tid + 256 * q;
            const int r = idx / NT, e = idx - r * NT;
            if (idx < TOT) bs[2 * ((r >> 1) + e * ES) + (r & 1)] = vals[q];
        }
    } else {
        for (int idx = tid; idx < 2 * LP * n; idx += nthr) {
            const int r = idx / n, e = idx - r * n;
            const long gl = line0 + r;
            T v = T(0);
            if (gl < nlines) {
                const long gi = gl * n + e;
                v = T(in[gi]);
                if (m1) v *= T(m1[gi]);
                if (m2) v *= T(m2[gi]);
            }
            bs[2 * ((r >> 1) + e * ES) + (r & 1)] = v;
        }
    }
    __syncthreads();
    C<T>* z = fft_any<T, -1, NT, LT, LT + 1>(b0, b1, LP, ES, plan, tw, tid, nthr);
    for (int idx = tid; idx < LP * kout; idx += nthr) {
        const int l = idx / kout, k = idx - l * kout;
        const long gl = line0 + 2 * l;
        if (gl >= nlines) continue;
        const C<T> zk = z[l + k * ES];
        const C<T> zm = z[l + ((n - k) % n) * ES];
        // X1 = (Z[k] + conj Z[n-k]) / 2 ;  X2 = (Z[k] - conj Z[n-k]) / (2i)
        const C<T> x1 = mk<T>(T(0.5) * (zk.x + zm.x), T(0.5) * (zk.y - zm.y));
        const C<T> x2 = mk<T>(T(0.5) * (zk.y + zm.y), T(-0.5) * (zk.x - zm.x));
        out[gl * kout + k] = x1;
        if (gl + 1 < nlines) out[(gl + 1) * kout + k] = x2;
    }
}

// z-pass, inverse (C2R): Hermitian half-lines X (kz < kin, zero above) of lines 2p, 2p+1 are packed as
// Z = X1 + i X2 over the full axis, inverse-transformed, and the real / imaginary parts written as the two
// real lines (times scale, times an optional pointwise multiplier).  As in a standard C2R the imaginary
// parts of the kz = 0 and kz = n/2 coefficients are ignored.
struct ZInvItem {
    const void* in;   // C<T>* [nlines][kin]
    void* out;        // T*    [nlines][n]
    int kin;
};
struct ZInvBatch {
    ZInvItem it[kMaxItems];
};

template <typename T, int NT = 0>
__global__ void __launch_bounds__(256) k_inv_z(ZInvBatch batch, long nlines, T scale, const T* __restrict__ mulout,
                                               FftPlan plan, const C<T>* __restrict__ twg, int LPrt) {
    extern __shared__ unsigned char smem_raw[];
    constexpr int LT = NT > 0 ? lines_per_cta_of<T>(NT) : 0;
    const ZInvItem item = batch.it[blockIdx.y];
    const C<T>* __restrict__ in = static_cast<const C<T>*>(item.in);
    T* __restrict__ out = static_cast<T*>(item.out);
    const int kin = item.kin;
    const int n = NT > 0 ? NT : plan.n;
    const int LP = NT > 0 ? LT : LPrt;
    const int ES = LP + 1;
    C<T>* b0 = reinterpret_cast<C<T>*>(smem_raw);
    C<T>* b1 = b0 + (size_t)n * ES;
    C<T>* tw = b1 + (size_t)n * ES;
    const long line0 = (long)blockIdx.x * 2 * LP;
    const int tid = threadIdx.x, nthr = blockDim.x;
    stage_twiddles<T>(tw, twg, n, tid, nthr);
    for (int idx = tid; idx < LP * n; idx += nthr) b0[idx % LP + (idx / LP) * ES] = mk<T>(T(0), T(0));
    __syncthreads();
    for (int idx = tid; idx < LP * kin; idx += nthr) {
        const int l = idx / kin, k = idx - l * kin;
        if (k > n / 2) continue;
        const long gl = line0 + 2 * l;
        C<T> x1 = mk<T>(T(0), T(0)), x2 = mk<T>(T(0), T(0));
        if (gl < nlines) x1 = in[gl * kin + k];
        if (gl + 1 < nlines) x2 = in[(gl + 1) * kin + k];
        if (k == 0 || 2 * k == n) {
            b0[l + k * ES] = mk<T>(x1.x, x2.x);
        } else {
            b0[l + k * ES] = mk<T>(x1.x - x2.y, x1.y + x2.x);
            b0[l + (n - k) * ES] = mk<T>(x1.x + x2.y, x2.x - x1.y);
        }
    }
    __syncthreads();
    C<T>* z = fft_any<T, +1, NT, LT, LT + 1>(b0, b1, LP, ES, plan, tw, tid, nthr);
    for (int idx = tid; idx < 2 * LP * n; idx += nthr) {
        const int r = idx / n, e = idx - r * n;
        const long gl = line0 + r;
        if (gl >= nlines) continue;
        const C<T> v = z[(r >> 1) + e * ES];
        T o = ((r & 1) ? v.y : v.x) * scale;
        if (mulout) o *= mulout[gl * n + e];
        out[gl * n + e] = o;
    }
}

// z-pass, inverse (C2R), length 512, register-resident: the same result as k_inv_z (including the packing of
// line pairs and the treatment of the kz = 0 and n/2 coefficients) computed as 512 = 8 x 8 x 8.  A group of 64
// threads transforms one packed line pair: thread t holds the eight points Z[t + 64 j]; stage 1 takes the 8-point
// DFT over j and multiplies by w512^(t k1); stage 2 (after an exchange through shared memory) the DFT over
// t2 = t / 8 and multiplies by w64^(t1 m1); stage 3 the DFT over t1 = t % 8, which leaves X[k1 + 8 m1 + 64 m2] in
// the thread; a last exchange through shared memory makes the 2 x 512 real outputs coalesced (16-byte stores).
// Twiddles are read once per thread from the table tw[m] = e^{-2 pi i m / 512} and kept in registers (measured:
// a shared-memory table costs more in bank conflicts than the registers it frees; prefetching the next pair's
// input costs more in occupancy than it hides).  Four groups per CTA, each synchronised by its own named barrier;
// a CTA takes `lpc` line pairs of one item (blockIdx.y).
// (immediate barrier ids, so that the kernel reserves 5 hardware barriers rather than all 16, which would cap the
// CTAs an SM can hold)
__device__ __forceinline__ void group_sync(int gid) {
    switch (gid) {
        case 0: asm volatile("bar.sync 1, 64;" ::: "memory"); break;
        case 1: asm volatile("bar.sync 2, 64;" ::: "memory"); break;
        case 2: asm volatile("bar.sync 3, 64;" ::: "memory"); break;
        default: asm volatile("bar.sync 4, 64;" ::: "memory"); break;
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_inv_z512(ZInvBatch batch, long nlines, T scale, const T* __restrict__ mulout,
                                                 const C<T>* __restrict__ twg, int lpc) {
    constexpr int N = 512, PAD = 9;                     // exchange rows of 8 complex values padded to 9
    constexpr int V = 16 / (int)sizeof(T);              // outputs per 16-byte vector store
    using VT = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
    __shared__ __align__(16) C<T> sbuf[4][64 * PAD];
    const ZInvItem item = batch.it[blockIdx.y];
    const C<T>* __restrict__ in = static_cast<const C<T>*>(item.in);
    T* __restrict__ out = static_cast<T*>(item.out);
    const int kin = item.kin;
    const int gid = threadIdx.x >> 6, t = threadIdx.x & 63;
    C<T>* buf = sbuf[gid];
    const int t1 = t & 7, k1s2 = t >> 3;                // stage-2 / stage-3 roles of this thread
    C<T> w1[8], w2[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        w1[r] = twg[(t * r) & (N - 1)];
        w2[r] = twg[(8 * t1 * r) & (N - 1)];
    }
    const long npairs = (nlines + 1) / 2;
    // stage-1 input of line pair p: Z[t + 64 j] of the packed Hermitian pair (zero beyond the kept wave numbers)
    auto load_pair = [&](long p, C<T> (&v)[8]) {
        const long l1 = 2 * p, l2 = 2 * p + 1;
        const C<T>* in1 = in + l1 * kin;
        const C<T>* in2 = in + l2 * kin;
        const bool has2 = l2 < nlines;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int k = t + 64 * j;
            C<T> z = mk<T>(T(0), T(0));
            if (k == 0 || 2 * k == N) {
                if (k < kin) z = mk<T>(in1[k].x, has2 ? in2[k].x : T(0));
            } else if (k < kin) {
                const C<T> a = in1[k];
                const C<T> b = has2 ? in2[k] : mk<T>(T(0), T(0));
                z = mk<T>(a.x - b.y, a.y + b.x);
            } else if (N - k < kin) {
                const C<T> a = in1[N - k];
                const C<T> b = has2 ? in2[N - k] : mk<T>(T(0), T(0));
                z = mk<T>(a.x + b.y, b.x - a.y);
            }
            v[j] = z;
        }
    };
    // the next pair's input is loaded before the current pair is transformed (global latency under the FFT)
    for (int q = gid; q < lpc; q += 4) {
        const long p = (long)blockIdx.x * lpc + q;
        if (p >= npairs) break;                          // uniform within the group
        const long l1 = 2 * p, l2 = 2 * p + 1;
        const bool has2 = l2 < nlines;
        C<T> v[8];
        load_pair(p, v);
        // stage 1: DFT over j, twiddle w512^(t k1) (inverse: conjugated table)
        dft<T, +1>(v, 8);
#pragma unroll
        for (int r = 1; r < 8; ++r) v[r] = mulc<T>(v[r], w1[r]);
#pragma unroll
        for (int r = 0; r < 8; ++r) buf[t * PAD + r] = v[r];
        group_sync(gid);
        // stage 2: thread (t1, k1) = (t % 8, t / 8) takes Y[t1 + 8 t2][k1], DFT over t2, twiddle w64^(t1 m1)
#pragma unroll
        for (int r = 0; r < 8; ++r) v[r] = buf[(t1 + 8 * r) * PAD + k1s2];
        dft<T, +1>(v, 8);
#pragma unroll
        for (int r = 1; r < 8; ++r) v[r] = mulc<T>(v[r], w2[r]);
        group_sync(gid);
#pragma unroll
        for (int r = 0; r < 8; ++r) buf[(k1s2 * 8 + r) * PAD + t1] = v[r];   // row (k1, m1), column t1
        group_sync(gid);
        // stage 3: thread w = (k1, m1) = (t / 8, t % 8) takes W[t1] for t1 = 0..7, DFT over t1 -> X[k1 + 8 m1 + 64 m2]
#pragma unroll
        for (int r = 0; r < 8; ++r) v[r] = buf[t * PAD + r];
        dft<T, +1>(v, 8);
        group_sync(gid);
        // outputs: real parts -> line l1, imaginary parts -> line l2, via shared memory for coalesced 16-byte stores
        T* re = reinterpret_cast<T*>(buf);
        T* im = re + N + 8;
        const int k1 = t >> 3, m1 = t & 7;
#pragma unroll
        for (int m2 = 0; m2 < 8; ++m2) {
            const int x = k1 + 8 * m1 + 64 * m2;
            re[x] = v[m2].x * scale;
            im[x] = v[m2].y * scale;
        }
        group_sync(gid);
        T* o1 = out + l1 * N;
        T* o2 = out + l2 * N;
#pragma unroll
        for (int e = 0; e < N / (64 * V); ++e) {
            const int x = V * (t + 64 * e);
            VT a = *reinterpret_cast<const VT*>(re + x);
            VT b = *reinterpret_cast<const VT*>(im + x);
            if (mulout) {
                T* pa = reinterpret_cast<T*>(&a);
                T* pb = reinterpret_cast<T*>(&b);
#pragma unroll
                for (int i = 0; i < V; ++i) {
                    pa[i] *= mulout[l1 * N + x + i];
                    if (has2) pb[i] *= mulout[l2 * N + x + i];
                }
            }
            *reinterpret_cast<VT*>(o1 + x) = a;
            if (has2) *reinterpret_cast<VT*>(o2 + x) = b;
        }
        group_sync(gid);
    }
}

// ------------------------------------------------------------------------------------------------
// z-pass, inverse (C2R), length 256, register-resident, one warp per packed line pair (the same result as k_inv_z,
// including the packing of line pairs and the kz = 0 and n/2 treatment; measured 44 us against the staged kernel's
// 46 us at 256^3 with 48 kept wave numbers; a forward counterpart on the same scheme was slower than k_fwd_z).  With k = t + 32 j and n = n1 + 8 n2,
// n2 = c + 8 d, t = a + 4 b (w_m = e^{DIR 2 pi i / m}):
//   X[n1 + 8 c + 64 d] = sum_a w4^(a d) [ w32^(a c) sum_b w8^(b c) ( w256^(t n1) sum_j Z[t + 32 j] w8^(j n1) ) ]
// stage 1: lane t takes the 8-point DFT over j of its points and the twiddles w256^(t n1); stage 2 (after an exchange
// through shared memory): lane (n1, a) = (lane / 4, lane % 4) the 8-point DFT over b and the twiddles w32^(a c);
// stage 3: lane (n1, c0) = (lane % 8, lane / 8) the two 4-point DFTs over a for c = c0 and c0 + 4.  Twiddles come
// from the table tw[m] = e^{-2 pi i m / 256} once per lane and stay in registers; the warp synchronises with
// __syncwarp only.  Eight warps a CTA; a CTA takes `lpc` line pairs.
constexpr int kZ256Pad = 9;   // exchange rows of 8 complex values padded to 9 (conflict-free column reads)

// In-register 256-point DFT of one warp (lane t holds v[j] = Z[t + 32 j]); on return lane (n1, c0) holds
// X[n1 + 8 c + 64 d] in v[d] (c = c0) and v[4 + d] (c = c0 + 4), n1 = lane % 8, c0 = lane / 8.
template <typename T, int DIR>
__device__ __forceinline__ void fft256_warp(C<T> (&v)[8], C<T>* buf, const C<T> (&w1)[8], const C<T> (&w2)[8],
                                            int lane) {
    dft<T, DIR>(v, 8);                                     // over j -> n1
#pragma unroll
    for (int r = 1; r < 8; ++r) v[r] = DIR < 0 ? mul<T>(v[r], w1[r]) : mulc<T>(v[r], w1[r]);
#pragma unroll
    for (int r = 0; r < 8; ++r) buf[lane * kZ256Pad + r] = v[r];          // row t, column n1
    __syncwarp();
    const int n1 = lane >> 2, a = lane & 3;
#pragma unroll
    for (int b = 0; b < 8; ++b) v[b] = buf[(a + 4 * b) * kZ256Pad + n1];  // Y[a + 4 b][n1]
    dft<T, DIR>(v, 8);                                     // over b -> c
#pragma unroll
    for (int r = 1; r < 8; ++r) v[r] = DIR < 0 ? mul<T>(v[r], w2[r]) : mulc<T>(v[r], w2[r]);
    __syncwarp();
#pragma unroll
    for (int c = 0; c < 8; ++c) buf[(n1 * 8 + c) * 4 + a] = v[c];          // [(n1, c)][a], 4 a row
    __syncwarp();
    const int m1 = lane & 7, c0 = lane >> 3;
    C<T> u[4], x[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) { u[q] = buf[(m1 * 8 + c0) * 4 + q]; x[q] = buf[(m1 * 8 + c0 + 4) * 4 + q]; }
    dft<T, DIR>(u, 4);                                     // over a -> d
    dft<T, DIR>(x, 4);
#pragma unroll
    for (int d = 0; d < 4; ++d) { v[d] = u[d]; v[4 + d] = x[d]; }
    __syncwarp();
}

template <typename T>
__device__ __forceinline__ void z256_twiddles(const C<T>* __restrict__ twg, int lane, C<T> (&w1)[8], C<T> (&w2)[8]) {
    const int a = lane & 3;
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        w1[r] = twg[(lane * r) & 255];
        w2[r] = twg[(8 * a * r) & 255];
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_inv_z256(ZInvBatch batch, long nlines, T scale, const T* __restrict__ mulout,
                                                 const C<T>* __restrict__ twg, int lpc) {
    constexpr int N = 256;
    __shared__ __align__(16) C<T> sbuf[8][32 * kZ256Pad];
    const ZInvItem item = batch.it[blockIdx.y];
    const C<T>* __restrict__ in = static_cast<const C<T>*>(item.in);
    T* __restrict__ out = static_cast<T*>(item.out);
    const int kin = item.kin;
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    C<T>* buf = sbuf[wid];
    C<T> w1[8], w2[8];
    z256_twiddles<T>(twg, lane, w1, w2);
    const long npairs = (nlines + 1) / 2;
    for (int q = wid; q < lpc; q += 8) {
        const long p = (long)blockIdx.x * lpc + q;
        if (p >= npairs) break;                          // uniform within the warp
        const long l1 = 2 * p, l2 = 2 * p + 1;
        const bool has2 = l2 < nlines;
        const C<T>* in1 = in + l1 * kin;
        const C<T>* in2 = in + l2 * kin;
        C<T> v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int k = lane + 32 * j;
            C<T> z = mk<T>(T(0), T(0));
            if (k == 0 || 2 * k == N) {
                if (k < kin) z = mk<T>(in1[k].x, has2 ? in2[k].x : T(0));
            } else if (k < kin) {
                const C<T> a = in1[k];
                const C<T> b = has2 ? in2[k] : mk<T>(T(0), T(0));
                z = mk<T>(a.x - b.y, a.y + b.x);
            } else if (N - k < kin) {
                const C<T> a = in1[N - k];
                const C<T> b = has2 ? in2[N - k] : mk<T>(T(0), T(0));
                z = mk<T>(a.x + b.y, b.x - a.y);
            }
            v[j] = z;
        }
        fft256_warp<T, +1>(v, buf, w1, w2, lane);
        // real parts -> line l1, imaginary parts -> line l2, through shared memory for coalesced stores
        T* re = reinterpret_cast<T*>(buf);
        T* im = re + N;
        const int m1 = lane & 7, c0 = lane >> 3;
#pragma unroll
        for (int d = 0; d < 4; ++d) {
            const int x0 = m1 + 8 * c0 + 64 * d, x1 = x0 + 32;
            re[x0] = v[d].x * scale;
            im[x0] = v[d].y * scale;
            re[x1] = v[4 + d].x * scale;
            im[x1] = v[4 + d].y * scale;
        }
        __syncwarp();
        T* o1 = out + l1 * N;
        T* o2 = out + l2 * N;
#pragma unroll
        for (int e = 0; e < N / 32; ++e) {
            const int x = lane + 32 * e;
            T a = re[x], b = im[x];
            if (mulout) {
                a *= mulout[l1 * N + x];
                if (has2) b *= mulout[l2 * N + x];
            }
            o1[x] = a;
            if (has2) o2[x] = b;
        }
        __syncwarp();
    }
}

// ------------------------------------------------------------------------------------------------
// z-pass, inverse (C2R), length 288 = 12 x 24, register-resident: the same result as k_inv_z (packing of line pairs,
// kz = 0 and n/2 treatment) as a two-stage Cooley-Tukey transform.  With k = t + 12 j and n = n1 + 24 n2,
//   z[n1 + 24 n2] = sum_t w12^(t n2) [ w288^(t n1) sum_j Z[t + 12 j] w24^(j n1) ]      (w_m = e^{+2 pi i / m}),
// so a group of 12 threads transforms one packed line pair: thread t takes the 24-point DFT over j of its points
// (in registers, as 3 x 8) and the twiddles w288^(t n1) (read once per thread from the table and kept in registers),
// the groups exchange through shared memory, and thread t takes the 12-point DFTs (as 3 x 4) of rows n1 = t and
// t + 12; a last exchange through shared memory makes the two real output lines coalesced (16-byte stores).  A CTA
// of 192 threads takes 16 line pairs per round and `ppc` line pairs of one item (blockIdx.y) in all.

// e^{i m pi / 12} for m = 0 .. 14 (multiples of 15 degrees; closed forms of cos / sin 15, 30, 45 degrees)
__host__ __device__ constexpr double root24_re(int m) {
    constexpr double c15 = 0.96592582628906829, s15 = 0.25881904510252076, c30 = 0.86602540378443865,
                     c45 = 0.70710678118654752;
    constexpr double t[15] = {1.0, c15, c30, c45, 0.5, s15, 0.0, -s15, -0.5, -c45, -c30, -c15, -1.0, -c15, -c30};
    return t[m];
}
__host__ __device__ constexpr double root24_im(int m) {
    constexpr double c15 = 0.96592582628906829, s15 = 0.25881904510252076, c30 = 0.86602540378443865,
                     c45 = 0.70710678118654752;
    constexpr double t[15] = {0.0, s15, 0.5, c45, c30, c15, 1.0, c15, c30, c45, 0.5, s15, 0.0, -s15, -0.5};
    return t[m];
}
// a * e^{DIR 2 pi i m / 24}
template <typename T, int DIR>
__device__ __forceinline__ C<T> rot24(C<T> a, int m) {
    const T c = T(root24_re(m)), s = T(DIR * root24_im(m));
    return mk<T>(a.x * c - a.y * s, a.x * s + a.y * c);
}

// X[n] = sum_j x[j] e^{DIR 2 pi i j n / 24}, natural order in and out: j = 3a + b, n = c + 8d.
template <typename T, int DIR>
__device__ __forceinline__ void dft24(C<T>* x) {
    C<T> A[3][8];
#pragma unroll
    for (int b = 0; b < 3; ++b) {
#pragma unroll
        for (int a = 0; a < 8; ++a) A[b][a] = x[3 * a + b];
        dft<T, DIR>(A[b], 8);
    }
#pragma unroll
    for (int b = 1; b < 3; ++b)
#pragma unroll
        for (int c = 1; c < 8; ++c) A[b][c] = rot24<T, DIR>(A[b][c], b * c);
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        C<T> y[3] = {A[0][c], A[1][c], A[2][c]};
        dft<T, DIR>(y, 3);
        x[c] = y[0];
        x[c + 8] = y[1];
        x[c + 16] = y[2];
    }
}

// X[n] = sum_j x[j] e^{DIR 2 pi i j n / 12}, natural order: j = 3a + b, n = c + 4d (w12^m = w24^(2m)).
template <typename T, int DIR>
__device__ __forceinline__ void dft12(C<T>* x) {
    C<T> A[3][4];
#pragma unroll
    for (int b = 0; b < 3; ++b) {
#pragma unroll
        for (int a = 0; a < 4; ++a) A[b][a] = x[3 * a + b];
        dft<T, DIR>(A[b], 4);
    }
#pragma unroll
    for (int b = 1; b < 3; ++b)
#pragma unroll
        for (int c = 1; c < 4; ++c) A[b][c] = rot24<T, DIR>(A[b][c], 2 * b * c);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        C<T> y[3] = {A[0][c], A[1][c], A[2][c]};
        dft<T, DIR>(y, 3);
        x[c] = y[0];
        x[c + 4] = y[1];
        x[c + 8] = y[2];
    }
}

// 16-byte and 8-byte asynchronous global -> shared copies (cp.async; completion by commit / wait_group).
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Copies the `bytes` (a multiple of 8) at src to dst with the CTA's threads: 16-byte pieces, then an 8-byte tail.
__device__ __forceinline__ void stage_block(unsigned char* dst, const unsigned char* src, long bytes, int tid, int nthr) {
    const long n16 = bytes >> 4;
    for (long i = tid; i < n16; i += nthr) cp_async16(dst + 16 * i, src + 16 * i);
    if ((bytes & 15) && tid == 0) cp_async8(dst + 16 * n16, src + 16 * n16);
    cp_async_commit();
}

constexpr int kZ288Threads = 192, kZ288Pairs = 16, kZ288Kmax = 145;
// exchange buffer of a group: 24 rows of 13 (row stride 13: the 12 threads of a group read 12 rows conflict-free),
// groups 316 float2 apart (316 = 12 mod 16: the two groups of a half-warp cover the 32 banks exactly)
constexpr int kZ288Rs = 13, kZ288Gs = 316;
// dynamic shared memory: twiddle table [288] float2, exchange buffers [16][316] float2, the staging barrier (16
// bytes), input stage [32 lines][kin] (16-byte aligned: (288 + 16 x 316) x 8 + 16 = 42768 bytes in)
inline size_t z288_smem(int kin_max) {
    return (size_t)(288 + kZ288Pairs * kZ288Gs + 2 + 2 * kZ288Pairs * kin_max) * sizeof(float2);
}

static __global__ void __launch_bounds__(192, 3) k_inv_z288(ZInvBatch batch, long nlines, float scale,
                                                           const float* __restrict__ mulout,
                                                           const float2* __restrict__ twg, int ppc, int* err) {
    constexpr int N = 288, TG = 12, P = 24, G = kZ288Pairs, RS = kZ288Rs, GS = kZ288Gs;
    static_assert((TG - 1) * (P - 1) < N, "twiddle index t n1 stays below N");
    extern __shared__ __align__(16) float2 z288_dyn[];
    float2* stw = z288_dyn;                           // e^{-2 pi i m / 288}
    float2* sbuf = z288_dyn + N;                      // exchange buffers
    uint64_t* sbar = reinterpret_cast<uint64_t*>(sbuf + G * GS);   // completion barrier of the staging copies
    float2* stage = sbuf + G * GS + 2;                // the round's input lines, [2 G][kin]
    const ZInvItem item = batch.it[blockIdx.y];
    const float2* __restrict__ in = static_cast<const float2*>(item.in);
    float* __restrict__ out = static_cast<float*>(item.out);
    const int kin = item.kin;                         // <= kin_max of the launch (<= 145, the Hermitian half)
    const int tid = threadIdx.x, g = tid / TG, t = tid - g * TG;
    float2* buf = sbuf + g * GS;
    for (int i = tid; i < N; i += kZ288Threads) stw[i] = twg[i];   // visible after the first round's barrier
    const long npairs = (nlines + 1) / 2;
    const long p_beg = (long)blockIdx.x * ppc;
    const long p_end = min(npairs, p_beg + ppc);
    // A round's input lines, 2q .. min(2 (q + G), nlines) - 1, are one contiguous block: with an even line count
    // (an even number of lines a round, 16 kin bytes a line pair) and a 16-byte aligned item, one bulk copy by the
    // TMA engine stages it (completion on sbar); otherwise every thread issues its share of 16-byte cp.async copies.
    const bool bulk = (nlines % 2 == 0) && (reinterpret_cast<uintptr_t>(in) & 15) == 0;
    uint32_t phase = 0;
    if (bulk && tid == 0) bulk_bar_init(sbar);
    __syncthreads();                                  // the barrier is initialised before its first use
    auto issue = [&](long q) {
        const long l0 = 2 * q, l1 = min(2 * min(q + G, p_end), nlines);
        const long bytes = (l1 - l0) * kin * (long)sizeof(float2);
        if (bulk) {
            if (tid == 0) bulk_g2s(stage, in + l0 * kin, (uint32_t)bytes, sbar);
        } else {
            stage_block(reinterpret_cast<unsigned char*>(stage), reinterpret_cast<const unsigned char*>(in + l0 * kin),
                        bytes, tid, kZ288Threads);
        }
    };
    if (p_beg < p_end) issue(p_beg);
    for (long p0 = p_beg; p0 < p_end; p0 += G) {
        const long p = p0 + g;
        const bool act = p < p_end;
        if (bulk) {
            // bounded wait for the round's copy; every thread takes the same decision (the barrier below)
            const bool landed = bulk_wait(sbar, phase, kBulkSpinLimit);
            phase ^= 1u;
            if (!__syncthreads_and(landed)) {
                if (tid == 0) {
                    atomicExch(err, 1);
                    bulk_wait(sbar, phase ^ 1u, kBulkSpinLimit);   // let the copy in flight land before exiting
                }
                return;
            }
        } else {
            cp_async_wait_all();
            __syncthreads();                          // the round's lines are in `stage`
        }
        float2 v[P];
        {
            const bool has2 = act && 2 * p + 1 < nlines;
            const float2* in1 = stage + (2 * g) * kin;
            const float2* in2 = in1 + kin;
#pragma unroll
            for (int j = 0; j < P; ++j) {
                const int k = t + TG * j;
                float2 z = make_float2(0.f, 0.f);
                if (act) {
                    if (k == 0 || 2 * k == N) {
                        if (k < kin) z = make_float2(in1[k].x, has2 ? in2[k].x : 0.f);
                    } else if (k < kin) {
                        const float2 a = in1[k];
                        const float2 b = has2 ? in2[k] : make_float2(0.f, 0.f);
                        z = make_float2(a.x - b.y, a.y + b.x);
                    } else if (N - k < kin) {
                        const float2 a = in1[N - k];
                        const float2 b = has2 ? in2[N - k] : make_float2(0.f, 0.f);
                        z = make_float2(a.x + b.y, b.x - a.y);
                    }
                }
                v[j] = z;
            }
        }
        __syncthreads();                              // every thread has its points: refill `stage`
        if (p0 + G < p_end) issue(p0 + G);
        // stage 1: 24-point DFT over j, twiddle w288^(t n1); rows n1 of the group's exchange buffer
        dft24<float, +1>(v);
        // twiddle w288^(t n1) = conj(tw[t n1]) (t n1 <= 11 x 23 < N: no reduction modulo N)
#pragma unroll
        for (int n1 = 1; n1 < P; ++n1) v[n1] = mulc<float>(v[n1], stw[t * n1]);
#pragma unroll
        for (int n1 = 0; n1 < P; ++n1) buf[n1 * RS + t] = v[n1];
        __syncthreads();
        // stage 2: 12-point DFTs over t of rows n1 = t and t + 12
        float2 o[2][TG];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
#pragma unroll
            for (int u = 0; u < TG; ++u) o[h][u] = buf[(t + 12 * h) * RS + u];
            dft12<float, +1>(o[h]);
        }
        __syncthreads();
        // outputs: z[n1 + 24 n2] -> real parts to line 2p, imaginary parts to line 2p + 1 (staged for coalescing)
        float* re = reinterpret_cast<float*>(buf);
        float* im = re + N;
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int n2 = 0; n2 < TG; ++n2) {
                const int n = t + 12 * h + 24 * n2;
                re[n] = o[h][n2].x * scale;
                im[n] = o[h][n2].y * scale;
            }
        __syncthreads();
        constexpr int Q = N / 4;                         // float4 per line
        for (int q = tid; q < G * 2 * Q; q += kZ288Threads) {
            const int gg = q / (2 * Q), r = q - gg * 2 * Q;
            const int side = r / Q, e4 = r - side * Q;
            const long pp = p0 + gg;
            const long l = 2 * pp + side;
            if (pp >= p_end || l >= nlines) continue;
            float4 a = *reinterpret_cast<const float4*>(reinterpret_cast<const float*>(sbuf + gg * GS) + side * N + 4 * e4);
            if (mulout) {
                const float* m = mulout + l * N + 4 * e4;
                a.x *= m[0]; a.y *= m[1]; a.z *= m[2]; a.w *= m[3];
            }
            *reinterpret_cast<float4*>(out + l * N + 4 * e4) = a;
        }
        // (the next round's first __syncthreads orders these reads of sbuf before its writes)
    }
    cp_async_wait_all();
}

// ------------------------------------------------------------------------------------------------
// Strided column pass (y or x axis).  Each CTA transforms TK consecutive columns of one outer slab.
//   forward (DIR = -1): input positions 0..n-1 at in[o*in_os + i*in_es + c]; keeps wave numbers
//                       f in out_rng, stored at out[o*out_os + (f - lo)*out_es + c].
//   inverse (DIR = +1): input holds wave numbers f = in_rng.lo + i (i < in_rng.cnt), zero elsewhere;
//                       all n positions are stored.
struct ColItem {
    const void* in;
    void* out;
    long in_os, in_es, out_os, out_es;
    int ncols, nouter;
    AxisRange rng;
};
struct ColBatch {
    ColItem it[kMaxItems];
};

template <typename T, int DIR, int NT = 0>
__global__ void __launch_bounds__(256) k_col(ColBatch batch, FftPlan plan, const C<T>* __restrict__ twg, int TKrt) {
    extern __shared__ unsigned char smem_raw[];
    constexpr int TT = NT > 0 ? cols_per_cta_of<T>(NT) : 0;
    const int TK = NT > 0 ? TT : TKrt;
    const ColItem item = batch.it[blockIdx.z];
    const int n = NT > 0 ? NT : plan.n;
    const int c0 = blockIdx.x * TK;
    const int o = blockIdx.y;
    if (c0 >= item.ncols || o >= item.nouter) return;
    const int nc = min(TK, item.ncols - c0);
    const C<T>* __restrict__ in = static_cast<const C<T>*>(item.in) + (long)o * item.in_os + c0;
    C<T>* __restrict__ out = static_cast<C<T>*>(item.out) + (long)o * item.out_os + c0;
    C<T>* b0 = reinterpret_cast<C<T>*>(smem_raw);
    C<T>* b1 = b0 + (size_t)n * TK;
    C<T>* tw = b1 + (size_t)n * TK;
    const int tid = threadIdx.x, nthr = blockDim.x;
    stage_twiddles<T>(tw, twg, n, tid, nthr);
    if constexpr (DIR < 0 && NT > 0) {
        // compile-time trip count (256 threads): all loads issued before the stores
        constexpr int IT = (NT * TT + 255) / 256;
        C<T> vals[IT];
#pragma unroll
        for (int q = 0; q < IT; ++q) {
            const int idx = tid + 256 * q;
            const int c = idx % TT, i = idx / TT;
            vals[q] = (idx < NT * TT && c < nc) ? in[(long)i * item.in_es + c] : mk<T>(T(0), T(0));
        }
#pragma unroll
        for (int q = 0; q < IT; ++q) {
            const int idx = tid + 256 * q;
            if (idx < NT * TT) b0[idx] = vals[q];
        }
    } else if constexpr (DIR < 0) {
        for (int idx = tid; idx < n * TK; idx += nthr) {
            const int c = idx % TK, i = idx / TK;
            b0[idx] = c < nc ? in[(long)i * item.in_es + c] : mk<T>(T(0), T(0));
        }
    } else if constexpr (NT > 0) {
        // compile-time bound on the kept rows (<= n): the loads are issued before the zero fill and the stores
        constexpr int IT = (NT * TT + 255) / 256;
        const int nld = item.rng.cnt * TT;
        C<T> vals[IT];
#pragma unroll
        for (int q = 0; q < IT; ++q) {
            const int idx = tid + 256 * q;
            const int c = idx % TT, i = idx / TT;
            vals[q] = (idx < nld && c < nc) ? in[(long)i * item.in_es + c] : mk<T>(T(0), T(0));
        }
        for (int idx = tid; idx < NT * TT; idx += 256) b0[idx] = mk<T>(T(0), T(0));
        __syncthreads();
#pragma unroll
        for (int q = 0; q < IT; ++q) {
            const int idx = tid + 256 * q;
            const int c = idx % TT, i = idx / TT;
            if (idx < nld && c < nc) b0[c + pos_of(item.rng.lo + i, NT) * TT] = vals[q];
        }
    } else {
        for (int idx = tid; idx < n * TK; idx += nthr) b0[idx] = mk<T>(T(0), T(0));
        __syncthreads();
        for (int idx = tid; idx < item.rng.cnt * TK; idx += nthr) {
            const int c = idx % TK, i = idx / TK;
            if (c < nc) b0[c + pos_of(item.rng.lo + i, n) * TK] = in[(long)i * item.in_es + c];
        }
    }
    __syncthreads();
    C<T>* z = fft_any<T, DIR, NT, TT, TT>(b0, b1, TK, TK, plan, tw, tid, nthr);
    if (DIR < 0) {
        for (int idx = tid; idx < item.rng.cnt * TK; idx += nthr) {
            const int c = idx % TK, i = idx / TK;
            if (c < nc) out[(long)i * item.out_es + c] = z[c + pos_of(item.rng.lo + i, n) * TK];
        }
    } else {
        for (int idx = tid; idx < n * TK; idx += nthr) {
            const int c = idx % TK, i = idx / TK;
            if (c < nc) out[(long)i * item.out_es + c] = z[idx];
        }
    }
}

// ------------------------------------------------------------------------------------------------
// Inverse y pass on 288-point columns (FP32), register-resident: the same two-stage transform as k_inv_z288
// (k = t + 12 j, n = n1 + 24 n2; a 24-point DFT over j, the twiddle w288^(t n1), a 12-point DFT over t), applied to
// complex columns.  A CTA of 192 threads takes 16 consecutive columns (wave numbers kz) of one x slab of one bin:
// thread (t, c) = (tid / 16, tid % 16) loads its 24 points straight from the bin's pruned input (rows = the bin's
// y wave numbers; zero outside them), so a warp reads and writes two rows of 16 consecutive columns (128 bytes
// each) at a time; the two stages exchange through shared memory (one 24 x 13 buffer a column).
constexpr int kY288Cols = 16, kY288Threads = 12 * kY288Cols;
// exchange buffers 313 float2 apart (>= 24 x 13; odd, so the 16 columns a half-warp touches fall on distinct bank
// pairs: 2 x 313 = 18 mod 32 words)
constexpr int kY288Gs = 313;
inline size_t y288_smem() { return (size_t)(288 + kY288Cols * kY288Gs) * sizeof(float2); }

static __global__ void __launch_bounds__(192, 3) k_inv_y288(ColBatch batch, const float2* __restrict__ twg) {
    constexpr int N = 288, TG = 12, P = 24, TC = kY288Cols, RS = kZ288Rs, GS = kY288Gs;
    static_assert(P * RS <= GS, "a column's exchange buffer holds 24 rows of 13");
    static_assert((TG - 1) * (P - 1) < N, "twiddle index t n1 stays below N");
    extern __shared__ __align__(16) float2 y288_dyn[];
    float2* stw = y288_dyn;                           // e^{-2 pi i m / 288}
    const ColItem item = batch.it[blockIdx.z];
    const int c0 = blockIdx.x * TC, o = blockIdx.y;
    if (c0 >= item.ncols || o >= item.nouter) return;   // uniform over the CTA
    const int tid = threadIdx.x, t = tid / TC, c = tid - t * TC;
    float2* buf = y288_dyn + N + c * GS;              // this column's exchange buffer
    for (int i = tid; i < N; i += kY288Threads) stw[i] = twg[i];
    const bool act = c0 + c < item.ncols;
    const float2* __restrict__ in = static_cast<const float2*>(item.in) + (long)o * item.in_os + c0 + c;
    float2* __restrict__ out = static_cast<float2*>(item.out) + (long)o * item.out_os + c0 + c;
    // points k = t + 12 j: wave number f = k (k < 144) or k - 288, input row f - lo when inside the bin's range
    float2 v[P];
#pragma unroll
    for (int j = 0; j < P; ++j) {
        const int k = t + TG * j;
        const int i = (k < N / 2 ? k : k - N) - item.rng.lo;
        v[j] = (act && i >= 0 && i < item.rng.cnt) ? in[(long)i * item.in_es] : make_float2(0.f, 0.f);
    }
    __syncthreads();                                  // the twiddle table is in place
    dft24<float, +1>(v);
#pragma unroll
    for (int n1 = 1; n1 < P; ++n1) v[n1] = mulc<float>(v[n1], stw[t * n1]);
#pragma unroll
    for (int n1 = 0; n1 < P; ++n1) buf[n1 * RS + t] = v[n1];
    __syncthreads();
    float2 w[2][TG];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
#pragma unroll
        for (int u = 0; u < TG; ++u) w[h][u] = buf[(t + 12 * h) * RS + u];
        dft12<float, +1>(w[h]);
    }
    if (!act) return;
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int n2 = 0; n2 < TG; ++n2) out[(long)(t + 12 * h + 24 * n2) * item.out_es] = w[h][n2];
}

// ------------------------------------------------------------------------------------------------
// First inverse pass with the shell filter: for bin b, columns are the (n_y, n_z) points of that bin's
// bounding box (flattened, n_z fastest); along x only wave numbers in the bin's x-range are loaded,
// each multiplied by Theta_b(|n|) (the bin's range of integer |n|^2), an optional per-mode weight
// (|n|^2-indexed table wtab, or the Legendre factor of the line of sight), and `scale`.
// spec == nullptr means a unit spectrum (the t_b maps that normalise the bispectrum).
constexpr int kLegendreM = 100;   // XInvItem::m of the global line of sight (weight L_ell(mu))
struct XInvItem {
    void* out;            // C<T>* [n0][ry.cnt * rz.cnt]
    AxisRange rx, ry, rz; // bin bounding box
    int bin;
    int slo, shi;         // the bin's range of integer |n|^2 (empty when slo > shi)
    int ell;              // 0: no weight; else L_ell(mu), mu = n_z / |n| (m == kLegendreM) or Ybar_lm(n / |n|)
    int m;
};
struct XInvBatch {
    XInvItem it[kMaxItems];
};

// Theta_b(|n|) x weight x scale x D(n) at the mode (fx, fy, fz) of the item's bin; false outside the bin.
template <typename T>
__device__ __forceinline__ bool x_filter_value(const XInvItem& item, const C<T>* __restrict__ spec, AxisRange gx,
                                               AxisRange gy, AxisRange gz, T scale, int fx, int fy, int fz, C<T>& v) {
    const int s = fx * fx + fy * fy + fz * fz;
    if (s < item.slo || s > item.shi) return false;
    T wgt = scale;
    if (item.ell && item.m == kLegendreM) {
        const T mu2 = T(fz * fz) / T(s);
        wgt *= item.ell == 2 ? T(0.5) * (T(3) * mu2 - T(1)) : (T(35) * mu2 * mu2 - T(30) * mu2 + T(3)) / T(8);
    } else if (item.ell) {
        const T inv = T(1) / sqrt(T(s));
        wgt *= ybar<T>(item.ell, item.m, T(fx) * inv, T(fy) * inv, T(fz) * inv);
    }
    v = mk<T>(wgt, T(0));
    if (spec) {
        const C<T> d = spec[(long)(fx - gx.lo) * ((long)gy.cnt * gz.cnt) + (long)(fy - gy.lo) * gz.cnt + (fz - gz.lo)];
        v = mk<T>(d.x * wgt, d.y * wgt);
    }
    return true;
}

template <typename T, int NT = 0>
__global__ void __launch_bounds__(256) k_inv_x_filter(XInvBatch batch, const C<T>* __restrict__ spec,
                                                      AxisRange gx, AxisRange gy, AxisRange gz, T scale,
                                                      FftPlan plan, const C<T>* __restrict__ twg, int TKrt) {
    extern __shared__ unsigned char smem_raw[];
    constexpr int TT = NT > 0 ? cols_per_cta_of<T>(NT) : 0;
    const int TK = NT > 0 ? TT : TKrt;
    const XInvItem item = batch.it[blockIdx.y];
    const int n = NT > 0 ? NT : plan.n;
    const int ncols = item.ry.cnt * item.rz.cnt;
    const int c0 = blockIdx.x * TK;
    if (c0 >= ncols) return;
    const int nc = min(TK, ncols - c0);
    C<T>* b0 = reinterpret_cast<C<T>*>(smem_raw);
    C<T>* b1 = b0 + (size_t)n * TK;
    C<T>* tw = b1 + (size_t)n * TK;
    const int tid = threadIdx.x, nthr = blockDim.x;
    stage_twiddles<T>(tw, twg, n, tid, nthr);
    // the filtered value of element idx (column c, x index i) and its shared-memory slot (-1: outside the bin)
    auto element = [&](int idx, C<T>& v) -> int {
        const int c = idx % TK, i = idx / TK;
        if (c >= nc) return -1;
        const int cc = c0 + c;
        const int fy = item.ry.lo + cc / item.rz.cnt;
        const int fz = item.rz.lo + cc % item.rz.cnt;
        const int fx = item.rx.lo + i;
        if (!x_filter_value<T>(item, spec, gx, gy, gz, scale, fx, fy, fz, v)) return -1;
        return c + pos_of(fx, n) * TK;
    };
    if constexpr (NT > 0) {
        // compile-time bound on the loaded elements (rx.cnt <= n): the spectrum loads are issued before the zero
        // fill and the stores
        constexpr int IT = (NT * TT + 255) / 256;
        static_assert(IT <= 32, "one validity bit an element");
        const int nld = item.rx.cnt * TT;
        C<T> vals[IT];
        unsigned keep = 0u;                               // element q lies in the bin (its slot is recomputed below)
#pragma unroll
        for (int q = 0; q < IT; ++q) {
            const int idx = tid + 256 * q;
            if (idx < nld && element(idx, vals[q]) >= 0) keep |= 1u << q;
        }
        for (int idx = tid; idx < NT * TT; idx += 256) b0[idx] = mk<T>(T(0), T(0));
        __syncthreads();
#pragma unroll
        for (int q = 0; q < IT; ++q) {
            if (!(keep >> q & 1u)) continue;
            const int idx = tid + 256 * q;
            b0[idx % TT + pos_of(item.rx.lo + idx / TT, NT) * TT] = vals[q];
        }
    } else {
        for (int idx = tid; idx < n * TK; idx += nthr) b0[idx] = mk<T>(T(0), T(0));
        __syncthreads();
        for (int idx = tid; idx < item.rx.cnt * TK; idx += nthr) {
            C<T> v;
            const int d = element(idx, v);
            if (d >= 0) b0[d] = v;
        }
    }
    __syncthreads();
    C<T>* z = fft_any<T, +1, NT, TT, TT>(b0, b1, TK, TK, plan, tw, tid, nthr);
    C<T>* __restrict__ out = static_cast<C<T>*>(item.out);
    for (int idx = tid; idx < n * TK; idx += nthr) {
        const int c = idx % TK, i = idx / TK;
        if (c < nc) out[(long)i * ncols + c0 + c] = z[idx];
    }
}

// The filter + x IFFT on 288-point x lines (FP32), register-resident like k_inv_y288: a CTA of 192 threads takes 16
// consecutive columns (points (n_y, n_z) of the bin's box, n_z fastest) of one bin; thread (t, c) forms its 24
// filtered points k = t + 12 j (wave number n_x = k or k - 288, zero outside the bin's x range and the bin) and
// takes the two-stage 288-point transform; rows of 16 consecutive columns are written (128 bytes).
static __global__ void __launch_bounds__(192, 3) k_inv_x288_filter(XInvBatch batch, const float2* __restrict__ spec,
                                                                  AxisRange gx, AxisRange gy, AxisRange gz,
                                                                  float scale, const float2* __restrict__ twg) {
    constexpr int N = 288, TG = 12, P = 24, TC = kY288Cols, RS = kZ288Rs, GS = kY288Gs;
    extern __shared__ __align__(16) float2 x288_dyn[];
    float2* stw = x288_dyn;                           // e^{-2 pi i m / 288}
    const XInvItem item = batch.it[blockIdx.y];
    const int ncols = item.ry.cnt * item.rz.cnt;
    const int c0 = blockIdx.x * TC;
    if (c0 >= ncols) return;                          // uniform over the CTA
    const int tid = threadIdx.x, t = tid / TC, c = tid - t * TC;
    float2* buf = x288_dyn + N + c * GS;
    for (int i = tid; i < N; i += kY288Threads) stw[i] = twg[i];
    const int cc = c0 + c;
    const bool act = cc < ncols;
    const int fy = act ? item.ry.lo + cc / item.rz.cnt : 0;
    const int fz = act ? item.rz.lo + cc % item.rz.cnt : 0;
    float2 v[P];
#pragma unroll
    for (int j = 0; j < P; ++j) {
        const int k = t + TG * j;
        const int fx = k < N / 2 ? k : k - N;
        const int i = fx - item.rx.lo;
        float2 x = make_float2(0.f, 0.f);          // stays zero outside the bin
        if (act && i >= 0 && i < item.rx.cnt) x_filter_value<float>(item, spec, gx, gy, gz, scale, fx, fy, fz, x);
        v[j] = x;
    }
    __syncthreads();                                  // the twiddle table is in place
    dft24<float, +1>(v);
#pragma unroll
    for (int n1 = 1; n1 < P; ++n1) v[n1] = mulc<float>(v[n1], stw[t * n1]);
#pragma unroll
    for (int n1 = 0; n1 < P; ++n1) buf[n1 * RS + t] = v[n1];
    __syncthreads();
    float2 w[2][TG];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
#pragma unroll
        for (int u = 0; u < TG; ++u) w[h][u] = buf[(t + 12 * h) * RS + u];
        dft12<float, +1>(w[h]);
    }
    if (!act) return;
    float2* __restrict__ out = static_cast<float2*>(item.out) + cc;
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int n2 = 0; n2 < TG; ++n2) out[(long)(t + 12 * h + 24 * n2) * ncols] = w[h][n2];
}

}  // namespace pb

namespace pb {
// Host-side dispatch of a launch over the compile-time lengths (NT = 0: run-time plan).
#define PB_WITH_NT(n, NTV, ...)                              \
    switch (n) {                                             \
        case 64: { constexpr int NTV = 64; __VA_ARGS__ } break;   \
        case 100: { constexpr int NTV = 100; __VA_ARGS__ } break; \
        case 128: { constexpr int NTV = 128; __VA_ARGS__ } break; \
        case 256: { constexpr int NTV = 256; __VA_ARGS__ } break; \
        case 512: { constexpr int NTV = 512; __VA_ARGS__ } break; \
        case 1024: { constexpr int NTV = 1024; __VA_ARGS__ } break; \
        default: { constexpr int NTV = 0; __VA_ARGS__ } break;    \
    }
// The inverse passes also run on the contraction grids (lengths 3m + 1 and up rounded to a 2-3-5 length):
// compile-time versions of the common ones (100: the masked 256^3 workload's bispectrum grid, whose B Fisher also
// takes forward transforms there).
#define PB_WITH_NT_INV(n, NTV, ...)                          \
    switch (n) {                                             \
        case 64: { constexpr int NTV = 64; __VA_ARGS__ } break;   \
        case 80: { constexpr int NTV = 80; __VA_ARGS__ } break;   \
        case 96: { constexpr int NTV = 96; __VA_ARGS__ } break;   \
        case 100: { constexpr int NTV = 100; __VA_ARGS__ } break; \
        case 128: { constexpr int NTV = 128; __VA_ARGS__ } break; \
        case 160: { constexpr int NTV = 160; __VA_ARGS__ } break; \
        case 192: { constexpr int NTV = 192; __VA_ARGS__ } break; \
        case 256: { constexpr int NTV = 256; __VA_ARGS__ } break; \
        case 288: { constexpr int NTV = 288; __VA_ARGS__ } break; \
        case 320: { constexpr int NTV = 320; __VA_ARGS__ } break; \
        case 512: { constexpr int NTV = 512; __VA_ARGS__ } break; \
        case 1024: { constexpr int NTV = 1024; __VA_ARGS__ } break; \
        default: { constexpr int NTV = 0; __VA_ARGS__ } break;    \
    }
}  // namespace pb
