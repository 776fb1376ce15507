// Triplet contraction M[(j<=k)][i] = sum_x g_j(x) g_k(x) h_i(x) over all grid cells x
// (the real-space sum of the separable bispectrum, Sec. 4.3.1 eq. beta-def; with h = g it gives
// S_abc for every a <= b and every c).  SIMT version: each CTA owns a range of cells and a group of
// pair rows; per chunk of CH cells it stages the maps in shared memory, forms the pair products once,
// and every thread accumulates a TM x TN register tile of outputs.
//
// Precision (float): products and chunk sums in FP32, flushed every FLUSH chunks into FP64 registers;
// per-CTA FP64 partials are reduced across CTAs in a fixed order (deterministic).
#pragma once
#include "common.cuh"

namespace pb {

constexpr int kCH = 32;       // cells per chunk
constexpr int kTM = 4;        // pair rows per thread
constexpr int kTN = 8;        // singles per thread
constexpr int kFlush = 16;    // chunks per FP32 partial sum (512 cells)

struct ContractGeom {
    int nb, nh, npairs;
    int rt, ct;        // thread tile grid (rt * ct <= 256)
    int rows_cta;      // pair rows per CTA (multiple of kTM)
    int nhp;           // padded singles (ct * kTN)
    int ngroups;       // row groups
    int ncb;           // cell blocks
    long cells_cta;    // cells per CTA (multiple of kCH)
};

template <typename T> struct Vec4;
template <> struct Vec4<float> {
    __device__ __forceinline__ static void load(const float* p, float* v) {
        float4 a = *reinterpret_cast<const float4*>(p);
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    }
};
template <> struct Vec4<double> {
    __device__ __forceinline__ static void load(const double* p, double* v) {
        double2 a = *reinterpret_cast<const double2*>(p);
        double2 b = *reinterpret_cast<const double2*>(p + 2);
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    }
};

template <typename T>
__global__ void __launch_bounds__(256) k_contract(const T* __restrict__ g, const T* __restrict__ h, long ncell,
                                                  const short2* __restrict__ pairs, ContractGeom G,
                                                  double* __restrict__ partial) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int tid = threadIdx.x;
    const int RP = G.rows_cta;
    const int NHP = G.nhp;
    const int GS = kCH + 1;
    T* sP = reinterpret_cast<T*>(smem_raw);          // [kCH][RP]
    T* sH = sP + (size_t)kCH * RP;                    // [kCH][NHP]
    T* sG = sH + (size_t)kCH * NHP;                   // [nb][GS]
    const int r0 = blockIdx.x * RP;
    const long cbeg = (long)blockIdx.y * G.cells_cta;
    const long cend = min(ncell, cbeg + G.cells_cta);
    const int rt = tid % G.rt, ct = tid / G.rt;
    const bool active = ct < G.ct && rt * kTM < RP;

    for (int idx = tid; idx < kCH * NHP; idx += blockDim.x) sH[idx] = T(0);

    T acc[kTM][kTN];
    double acc64[kTM][kTN];
#pragma unroll
    for (int u = 0; u < kTM; ++u)
#pragma unroll
        for (int v = 0; v < kTN; ++v) { acc[u][v] = T(0); acc64[u][v] = 0.0; }

    int chunk = 0;
    for (long c0 = cbeg; c0 < cend; c0 += kCH, ++chunk) {
        __syncthreads();
        for (int idx = tid; idx < G.nb * kCH; idx += blockDim.x) {
            const int b = idx / kCH, x = idx - b * kCH;
            const long cell = c0 + x;
            sG[b * GS + x] = cell < cend ? g[(long)b * ncell + cell] : T(0);
        }
        if (h) {
            for (int idx = tid; idx < G.nh * kCH; idx += blockDim.x) {
                const int i = idx / kCH, x = idx - i * kCH;
                const long cell = c0 + x;
                sH[x * NHP + i] = cell < cend ? h[(long)i * ncell + cell] : T(0);
            }
        }
        __syncthreads();
        if (!h) {
            for (int idx = tid; idx < G.nh * kCH; idx += blockDim.x) {
                const int x = idx % kCH, i = idx / kCH;
                sH[x * NHP + i] = sG[i * GS + x];
            }
        }
        for (int idx = tid; idx < RP * kCH; idx += blockDim.x) {
            const int p = idx % RP, x = idx / RP;
            const int gp = r0 + p;
            T v = T(0);
            if (gp < G.npairs) {
                const short2 jk = pairs[gp];
                v = sG[jk.x * GS + x] * sG[jk.y * GS + x];
            }
            sP[x * RP + p] = v;
        }
        __syncthreads();
        if (active) {
#pragma unroll 4
            for (int x = 0; x < kCH; ++x) {
                T a[kTM], b[kTN];
                Vec4<T>::load(sP + x * RP + rt * kTM, a);
                Vec4<T>::load(sH + x * NHP + ct * kTN, b);
                Vec4<T>::load(sH + x * NHP + ct * kTN + 4, b + 4);
#pragma unroll
                for (int u = 0; u < kTM; ++u)
#pragma unroll
                    for (int v = 0; v < kTN; ++v) acc[u][v] = fma(a[u], b[v], acc[u][v]);
            }
            if ((chunk + 1) % kFlush == 0) {
#pragma unroll
                for (int u = 0; u < kTM; ++u)
#pragma unroll
                    for (int v = 0; v < kTN; ++v) { acc64[u][v] += (double)acc[u][v]; acc[u][v] = T(0); }
            }
        }
    }
    if (!active) return;
    double* out = partial + (size_t)blockIdx.y * G.npairs * G.nh;
#pragma unroll
    for (int u = 0; u < kTM; ++u) {
        const int gp = r0 + rt * kTM + u;
        if (gp >= G.npairs) continue;
#pragma unroll
        for (int v = 0; v < kTN; ++v) {
            const int i = ct * kTN + v;
            if (i < G.nh) out[(size_t)gp * G.nh + i] = acc64[u][v] + (double)acc[u][v];
        }
    }
}

// Sum per-cell-block partials in a fixed order: out[o] = sum_cb partial[cb][o].
static __global__ void k_reduce_partials(const double* __restrict__ partial, int ncb, long nout, double* __restrict__ out) {
    const long o = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= nout) return;
    double s = 0.0;
    for (int cb = 0; cb < ncb; ++cb) s += partial[(size_t)cb * nout + o];
    out[o] = s;
}

// ------------------------------------------------------------------------------------------------
// P_ell binning reduction (Sec. 3.4.1, eq. pk-limit): num[ell][b] = sum_{k in b} L_ell(mu) |D(k)|^2 over
// the full k-grid, evaluated on the half spectrum with coefficient w_k L_ell (w_k = 1 on the kz = 0 and
// Nyquist planes, 2 elsewhere) precomputed per mode in FP64.  One CTA per (bin, segment of that bin's
// mode list); deterministic tree reduction in FP64.
template <typename T>
__global__ void __launch_bounds__(256) k_pk_bin(const C<T>* __restrict__ spec, const int* __restrict__ offs,
                                                const double* __restrict__ coef, long nmodes_total,
                                                const int* __restrict__ bin_start, int nell, int seg_len,
                                                double* __restrict__ partial /*[nb][nseg][nell]*/) {
    __shared__ double red[256 * 3];
    const int b = blockIdx.x, seg = blockIdx.y;
    const long beg = bin_start[b] + (long)seg * seg_len;
    const long end = min((long)bin_start[b + 1], beg + seg_len);
    double s[3] = {0.0, 0.0, 0.0};
    for (long m = beg + threadIdx.x; m < end; m += blockDim.x) {
        const C<T> d = spec[offs[m]];
        const double p = (double)d.x * (double)d.x + (double)d.y * (double)d.y;
        for (int l = 0; l < nell; ++l) s[l] += coef[(long)l * nmodes_total + m] * p;
    }
    for (int l = 0; l < 3; ++l) red[l * 256 + threadIdx.x] = s[l];
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int l = 0; l < 3; ++l) red[l * 256 + threadIdx.x] += red[l * 256 + threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < nell) partial[((long)b * gridDim.y + seg) * nell + threadIdx.x] = red[threadIdx.x * 256];
}

}  // namespace pb
