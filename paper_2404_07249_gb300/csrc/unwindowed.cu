// Masked ("unwindowed") estimators with a global line of sight: FKP weighting (Sec. 2.4, eq. Sinv-fkp), the
// power-spectrum numerator and Monte Carlo Fisher matrix (Sec. 3.3, eqs. pk-num-fft, Q-alpha-global,
// fish-from-Q), the bispectrum numerator with its Monte Carlo linear term (Sec. 4.3.2, eq.
// b-numerator-practical), the bispectrum Q-derivatives and Monte Carlo Fisher matrix (Sec. 4.3.4, eqs.
// Q-bis-global, bk-fish-def) and the FP64 solves x = F^-1 x_num (eqs. pk-estimator-def, bk-estimator-def).
//
// Data model: d = n delta (pixel window m = 1, no noise); S^-1 = w (diagonal); S^-1 P = w n.  Monte Carlo maps
// are unit Gaussian white noise (A = I) from Philox4x32-10 + Box-Muller (Salmon et al., SC'11), generated on
// the device with the same counter layout as the test oracle: map `draw` of `stream` has at flat cell i the
// value z_{i mod 4} of block j = i / 4, key = (seed lo, seed hi), counter = (j lo, j hi, draw, stream).
// Streams: 0, 1 = the pair (a1, a2) of the bispectrum Fisher; 2 = the power-spectrum Fisher draws.
// Everything is in pixel units (cell volume 1); physical units: P = p V / N, B = b (V / N)^2.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "polybin_internal.h"

namespace pb {
namespace uw {

// ---------------------------------------------------------------------------------------------- kernels

// w = 1 / (n P_FKP + 1), evaluated in FP64 and stored in the working precision.
template <typename T>
__global__ void k_fkp(const float* __restrict__ n, double p0, T* __restrict__ w, long N) {
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long)gridDim.x * blockDim.x)
        w[i] = (T)(1.0 / ((double)n[i] * p0 + 1.0));
}

__device__ __forceinline__ void philox_round(uint32_t& c0, uint32_t& c1, uint32_t& c2, uint32_t& c3, uint32_t k0,
                                             uint32_t k1) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t hi0 = __umulhi(M0, c0), lo0 = M0 * c0;
    const uint32_t hi1 = __umulhi(M1, c2), lo1 = M1 * c2;
    const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
}

// Gaussian white-noise map (Philox4x32-10 + Box-Muller in FP64).
template <typename T>
__global__ void k_draw(T* __restrict__ out, long N, unsigned long long seed, uint32_t draw, uint32_t stream) {
    const long nblk = (N + 3) / 4;
    for (long j = (long)blockIdx.x * blockDim.x + threadIdx.x; j < nblk; j += (long)gridDim.x * blockDim.x) {
        uint32_t c0 = (uint32_t)j, c1 = (uint32_t)((unsigned long long)j >> 32), c2 = draw, c3 = stream;
        uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
#pragma unroll
        for (int r = 0; r < 10; ++r) {
            if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
            philox_round(c0, c1, c2, c3, k0, k1);
        }
        const double t = 2.3283064365386963e-10;  // 2^-32
        const double u0 = ((double)c0 + 0.5) * t, u1 = ((double)c1 + 0.5) * t;
        const double u2 = ((double)c2 + 0.5) * t, u3 = ((double)c3 + 0.5) * t;
        const double r01 = sqrt(-2.0 * log(u0)), r23 = sqrt(-2.0 * log(u2));
        double s1, co1, s3, co3;
        sincospi(2.0 * u1, &s1, &co1);
        sincospi(2.0 * u3, &s3, &co3);
        const double z[4] = {r01 * co1, r01 * s1, r23 * co3, r23 * s3};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const long i = 4 * j + q;
            if (i < N) out[i] = (T)z[q];
        }
    }
}

// Binned cross products over the half spectrum: out[b][seg][ell] = sum_{modes m of bin b} coef_ell(m) Re(conj X A).
template <typename T>
__global__ void __launch_bounds__(256) k_cross_bin(const C<T>* __restrict__ X, const C<T>* __restrict__ A,
                                                   const int* __restrict__ offs, const double* __restrict__ coef,
                                                   long nmodes_total, const int* __restrict__ bin_start, int nell,
                                                   int seg_len, double* __restrict__ partial) {
    __shared__ double red[256 * 3];
    const int b = blockIdx.x, seg = blockIdx.y;
    const long beg = bin_start[b] + (long)seg * seg_len;
    const long end = min((long)bin_start[b + 1], beg + seg_len);
    double s[3] = {0.0, 0.0, 0.0};
    for (long m = beg + threadIdx.x; m < end; m += blockDim.x) {
        const C<T> x = X[offs[m]], a = A[offs[m]];
        const double p = (double)x.x * (double)a.x + (double)x.y * (double)a.y;
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

// Q-derivative spectrum of one triplet (a, b, c) from the pair spectra of two fields (eq. Q-bis-global):
//   out(k) = fac [ Theta_c (P1_ab - P2_ab) + Theta_a (P1_bc - P2_bc) + Theta_b (P1_ac - P2_ac) ](k),
// fac = 2 / Delta_abc, over every entry of the box (zero outside bins a, b, c).
template <typename T>
__global__ void k_qcomb(const C<T>* __restrict__ P1, const C<T>* __restrict__ P2, long pab, long pbc, long pac,
                        int a, int b, int c, T fac, AxisRange gx, AxisRange gy, AxisRange gz,
                        const int16_t* __restrict__ lut, int smax, C<T>* __restrict__ out) {
    const long nbox = (long)gx.cnt * gy.cnt * gz.cnt;
    for (long o = (long)blockIdx.x * blockDim.x + threadIdx.x; o < nbox; o += (long)gridDim.x * blockDim.x) {
        const int iz = (int)(o % gz.cnt);
        const long r = o / gz.cnt;
        const int iy = (int)(r % gy.cnt), ix = (int)(r / gy.cnt);
        const int fx = gx.lo + ix, fy = gy.lo + iy, fz = gz.lo + iz;
        const int s = fx * fx + fy * fy + fz * fz;
        const int bin = (s <= smax) ? lut[s] : -1;
        T re = T(0), im = T(0);
        if (bin >= 0) {
            if (bin == c) { const C<T> u = P1[pab + o], v = P2[pab + o]; re += u.x - v.x; im += u.y - v.y; }
            if (bin == a) { const C<T> u = P1[pbc + o], v = P2[pbc + o]; re += u.x - v.x; im += u.y - v.y; }
            if (bin == b) { const C<T> u = P1[pac + o], v = P2[pac + o]; re += u.x - v.x; im += u.y - v.y; }
        }
        out[o] = mk<T>(fac * re, fac * im);
    }
}

// Compact copy of the binned modes of a box spectrum: out[m] = box[offs[m]] (times wm[m] when wm is not NULL: the
// half-spectrum weight, 1 or 2, exact in any precision).
template <typename T>
__global__ void k_gather(const C<T>* __restrict__ box, const int* __restrict__ offs, long M, C<T>* __restrict__ out,
                         const double* __restrict__ wm = nullptr) {
    for (long m = (long)blockIdx.x * blockDim.x + threadIdx.x; m < M; m += (long)gridDim.x * blockDim.x) {
        const C<T> v = box[offs[m]];
        out[m] = wm ? mk<T>(v.x * (T)wm[m], v.y * (T)wm[m]) : v;
    }
}

// out[i][j] += scale * sum_m w_m Re(conj(Z[i][m]) Y[j][m])   (FP64 accumulation; 32 x 32 tile per CTA).
template <typename T>
__global__ void __launch_bounds__(256) k_gram(const C<T>* __restrict__ Z, const C<T>* __restrict__ Y,
                                              const double* __restrict__ wm, int nA, int nB, long M, long ld,
                                              double scale, double* __restrict__ out) {
    __shared__ double sz[32][65];   // 64 used (re, im interleaved) + 1 pad: conflict-free row access
    __shared__ double sy[32][65];
    const int i0 = blockIdx.x * 32, j0 = blockIdx.y * 32;
    const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;   // ty in [0, 8): 4 rows each
    double acc[4] = {0, 0, 0, 0};
    for (long m0 = 0; m0 < M; m0 += 32) {
        for (int q = threadIdx.x; q < 32 * 32; q += 256) {
            const int r = q / 32, k = q % 32;
            const long m = m0 + k;
            C<T> z = mk<T>(T(0), T(0)), y = mk<T>(T(0), T(0));
            double wk = 0.0;
            if (m < M) {
                wk = wm[m];
                if (i0 + r < nA) z = Z[(long)(i0 + r) * ld + m];
                if (j0 + r < nB) y = Y[(long)(j0 + r) * ld + m];
            }
            sz[r][2 * k] = wk * (double)z.x;
            sz[r][2 * k + 1] = wk * (double)z.y;
            sy[r][2 * k] = (double)y.x;
            sy[r][2 * k + 1] = (double)y.y;
        }
        __syncthreads();
        for (int k = 0; k < 64; ++k) {
            const double yv = sy[tx][k];
#pragma unroll
            for (int u = 0; u < 4; ++u) acc[u] += sz[ty * 4 + u][k] * yv;
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int i = i0 + ty * 4 + u, j = j0 + tx;
        if (i < nA && j < nB) out[(long)i * nB + j] += scale * acc[u];
    }
}

// Dense FP64 LU with partial pivoting and solve, one CTA: A (n x n, row major) is overwritten by its factors,
// B (n x nrhs, row major) by the solution.  info = 0, or k + 1 if the pivot of column k is exactly zero.
__global__ void __launch_bounds__(1024) k_lu_solve(double* __restrict__ A, int n, double* __restrict__ B, int nrhs,
                                                   int* __restrict__ info) {
    __shared__ double sval[1024];
    __shared__ int sidx[1024];
    __shared__ int piv;
    const int tid = threadIdx.x, nt = blockDim.x;
    if (tid == 0) *info = 0;
    for (int k = 0; k < n; ++k) {
        double best = -1.0;
        int bi = k;
        for (int i = k + tid; i < n; i += nt) {
            const double v = fabs(A[(long)i * n + k]);
            if (v > best) { best = v; bi = i; }
        }
        sval[tid] = best;
        sidx[tid] = bi;
        __syncthreads();
        for (int w = nt / 2; w > 0; w >>= 1) {
            if (tid < w && (sval[tid + w] > sval[tid] || (sval[tid + w] == sval[tid] && sidx[tid + w] < sidx[tid]))) {
                sval[tid] = sval[tid + w];
                sidx[tid] = sidx[tid + w];
            }
            __syncthreads();
        }
        if (tid == 0) {
            piv = sidx[0];
            if (sval[0] == 0.0 && *info == 0) *info = k + 1;
        }
        __syncthreads();
        const int p = piv;
        if (p != k) {
            for (int j = tid; j < n; j += nt) {
                const double t = A[(long)k * n + j]; A[(long)k * n + j] = A[(long)p * n + j]; A[(long)p * n + j] = t;
            }
            for (int j = tid; j < nrhs; j += nt) {
                const double t = B[(long)k * nrhs + j]; B[(long)k * nrhs + j] = B[(long)p * nrhs + j]; B[(long)p * nrhs + j] = t;
            }
        }
        __syncthreads();
        const double d = A[(long)k * n + k];
        if (d != 0.0)
            for (int i = k + 1 + tid; i < n; i += nt) A[(long)i * n + k] /= d;
        __syncthreads();
        const int rows = n - k - 1, cols = n - k - 1;
        for (long q = tid; q < (long)rows * cols; q += nt) {
            const int i = k + 1 + (int)(q / cols), j = k + 1 + (int)(q % cols);
            A[(long)i * n + j] -= A[(long)i * n + k] * A[(long)k * n + j];
        }
        for (long q = tid; q < (long)rows * nrhs; q += nt) {
            const int i = k + 1 + (int)(q / nrhs), j = (int)(q % nrhs);
            B[(long)i * nrhs + j] -= A[(long)i * n + k] * B[(long)k * nrhs + j];
        }
        __syncthreads();
    }
    // back substitution U x = y, column by column of the right-hand sides
    for (int k = n - 1; k >= 0; --k) {
        const double d = A[(long)k * n + k];
        for (int j = tid; j < nrhs; j += nt) B[(long)k * nrhs + j] = d != 0.0 ? B[(long)k * nrhs + j] / d : NAN;
        __syncthreads();
        for (long q = tid; q < (long)k * nrhs; q += nt) {
            const int i = (int)(q / nrhs), j = (int)(q % nrhs);
            B[(long)i * nrhs + j] -= A[(long)i * n + k] * B[(long)k * nrhs + j];
        }
        __syncthreads();
    }
}

// y = M x (FP64), M n x n row major.
__global__ void k_gemv(const double* __restrict__ M, const double* __restrict__ x, int n, double* __restrict__ y) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double s = 0.0;
    for (int j = 0; j < n; ++j) s += M[(long)i * n + j] * x[j];
    y[i] = s;
}

// ---- local (Yamamoto) line of sight: real harmonics Ybar_lm of the cell direction and of the wave vector

// Cell geometry of the data grid: spacing h, half box, observer (box coordinates centred on the origin).
template <typename T>
struct CellGeom {
    int N[3];
    T h[3], half_l, obs[3];
};

// out[i] = Ybar_lm(x_i) in[i] (times m1[i] m2[i] when given), x_i the direction of cell i from the observer.
template <typename T, typename TIN, typename TM>
__global__ void k_mul_ylm(const TIN* __restrict__ in, const TM* __restrict__ m1, const TM* __restrict__ m2,
                          T* __restrict__ out, int ell, int m, CellGeom<T> cg) {
    const long n = (long)cg.N[0] * cg.N[1] * cg.N[2];
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        // 32-bit unsigned index arithmetic (N < 2^31): 64-bit division per cell dominated these kernels
        const unsigned ui = (unsigned)i, n2 = (unsigned)cg.N[2], n1 = (unsigned)cg.N[1];
        const unsigned r = ui / n2, k = ui - r * n2;
        const unsigned a = r / n1, j = r - a * n1;
        T x, y, z;
        cell_direction<T>(a, j, k, cg.h, cg.half_l, cg.obs, x, y, z);
        T v = ybar<T>(ell, m, x, y, z) * T(in[i]);
        if (m1) v *= T(m1[i]);
        if (m2) v *= T(m2[i]);
        out[i] = v;
    }
}

// Q[b][i] += fac Ybar_lm(x_i) q[b][i] for the nb maps (one harmonic evaluation a cell).
template <typename T>
__global__ void k_ylm_axpy(T* __restrict__ Q, const T* __restrict__ q, int nb, int ell, int m, T fac, CellGeom<T> cg) {
    const long n = (long)cg.N[0] * cg.N[1] * cg.N[2];
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        // 32-bit unsigned index arithmetic (N < 2^31): 64-bit division per cell dominated these kernels
        const unsigned ui = (unsigned)i, n2 = (unsigned)cg.N[2], n1 = (unsigned)cg.N[1];
        const unsigned r = ui / n2, k = ui - r * n2;
        const unsigned a = r / n1, j = r - a * n1;
        T x, y, z;
        cell_direction<T>(a, j, k, cg.h, cg.half_l, cg.obs, x, y, z);
        const T yv = fac * ybar<T>(ell, m, x, y, z);
        for (int b = 0; b < nb; ++b) Q[(size_t)b * n + i] += yv * q[(size_t)b * n + i];
    }
}

// Direction of box entry o (wave numbers gx.lo + ix, gy.lo + iy, iz); false at n = 0.
__device__ __forceinline__ bool box_direction(long o, AxisRange gx, AxisRange gy, AxisRange gz, double& x, double& y,
                                              double& z) {
    const int iz = (int)(o % gz.cnt);
    const long r = o / gz.cnt;
    const int iy = (int)(r % gy.cnt), ix = (int)(r / gy.cnt);
    const double fx = gx.lo + ix, fy = gy.lo + iy, fz = gz.lo + iz;
    const double s = fx * fx + fy * fy + fz * fz;
    if (s <= 0) return false;
    const double inv = 1.0 / sqrt(s);
    x = fx * inv; y = fy * inv; z = fz * inv;
    return true;
}

// H[o] (= or +=) Ybar_lm(k_o) G[o] over the box (FP64 harmonic, working-precision product).
template <typename T>
__global__ void k_ylm_box_accum(const C<T>* __restrict__ G, C<T>* __restrict__ H, int ell, int m, int first,
                                AxisRange gx, AxisRange gy, AxisRange gz) {
    const long nbox = (long)gx.cnt * gy.cnt * gz.cnt;
    for (long o = (long)blockIdx.x * blockDim.x + threadIdx.x; o < nbox; o += (long)gridDim.x * blockDim.x) {
        double x, y, z;
        const T yv = box_direction(o, gx, gy, gz, x, y, z) ? (T)ybar<double>(ell, m, x, y, z) : T(0);
        const C<T> g = G[o];
        const C<T> v = mk<T>(yv * g.x, yv * g.y);
        H[o] = first ? v : add<T>(H[o], v);
    }
}

// acc[q] (= or +=) Ybar_lm(k_q) box[offs[q]] over the binned modes (FP64 accumulation).
template <typename T>
__global__ void k_ylm_gather(const C<T>* __restrict__ box, const int* __restrict__ offs, long M, int ell, int m,
                             int first, AxisRange gx, AxisRange gy, AxisRange gz, double2* __restrict__ acc) {
    for (long q = (long)blockIdx.x * blockDim.x + threadIdx.x; q < M; q += (long)gridDim.x * blockDim.x) {
        const long o = offs[q];
        double x, y, z;
        const double yv = box_direction(o, gx, gy, gz, x, y, z) ? ybar<double>(ell, m, x, y, z) : 0.0;
        const C<T> g = box[o];
        const double2 v = make_double2(yv * (double)g.x, yv * (double)g.y);
        acc[q] = first ? v : make_double2(acc[q].x + v.x, acc[q].y + v.y);
    }
}

// out[b][seg][l] = sum_{binned modes q of bin b} w_q Re(conj(X[offs[q]]) Y[l][q])  (w_q = 1 or 2: the half spectrum).
template <typename T>
__global__ void __launch_bounds__(256) k_cross_bin_local(const C<T>* __restrict__ X, const double2* __restrict__ Y,
                                                         const int* __restrict__ offs, const double* __restrict__ wq,
                                                         long M, const int* __restrict__ bin_start, int nell,
                                                         int seg_len, double* __restrict__ partial) {
    __shared__ double red[256 * 3];
    const int b = blockIdx.x, seg = blockIdx.y;
    const long beg = bin_start[b] + (long)seg * seg_len;
    const long end = min((long)bin_start[b + 1], beg + seg_len);
    double s[3] = {0.0, 0.0, 0.0};
    for (long q = beg + threadIdx.x; q < end; q += blockDim.x) {
        const C<T> x = X[offs[q]];
        for (int l = 0; l < nell; ++l) {
            const double2 y = Y[(long)l * M + q];
            s[l] += wq[q] * ((double)x.x * y.x + (double)x.y * y.y);
        }
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

// out = scale a (b) m: the noise-weighted products N3[a1, a2] = n3 a1 a2 / V^2 and N2 a = d2 a / V.
template <typename T>
__global__ void k_noise_map(T* __restrict__ out, const T* __restrict__ a, const T* __restrict__ b,
                            const float* __restrict__ m, T scale, long N) {
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long)gridDim.x * blockDim.x) {
        T v = a[i] * T(m[i]) * scale;
        if (b) v *= b[i];
        out[i] = v;
    }
}

}  // namespace uw

// ---------------------------------------------------------------------------------------------- state

struct UwState {
    size_t elem = 0;
    void* g2 = nullptr;       // second set of shell maps [nb][N]
    void* xmap = nullptr;     // one real map [N]
    void* a[2] = {nullptr, nullptr};  // Monte Carlo maps
    void* spec[4] = {nullptr, nullptr, nullptr, nullptr};  // box spectra
    void* pairs = nullptr;    // pair spectra [4][npairs][box]
    void* qbox = nullptr;     // one box spectrum
    void* zc = nullptr;       // compact [nt][M]
    void* yc = nullptr;       // compact [nt][M]
    void* v1 = nullptr;       // inverse-from-box intermediates [N0][By][Bz]
    void* v2 = nullptr;       //                                [N0][N1][Bz]
    double* dF = nullptr;     // device Fisher accumulator
    double* dpart = nullptr;  // cross-bin partials
    double* dvec = nullptr;
    double* dvec2 = nullptr;
    int* dinfo = nullptr;
    std::vector<double> Fp, Fb, Fp_inv, Fb_inv;   // host copies
    double* dFp_inv = nullptr;
    double* dFb_inv = nullptr;
    bool have_p = false, have_b = false;
    // local line of sight: compact sum_m Ybar_lm(k) FT[Ybar_lm u](k) per ell [3][M]; a box of the same sums; nb maps of
    // one harmonic's inverse transforms; the Fisher matrix and its inverse
    double2* ylc = nullptr;
    void* hbox = nullptr;
    void* g3 = nullptr;
    std::vector<double> Fl, Fl_inv;
    double* dFl_inv = nullptr;
    bool have_l = false;
    // optimal weighting: the Fisher matrix, its inverse and the weighting it was computed with
    std::vector<double> Fo, Fo_inv;
    double* dFo_inv = nullptr;
    bool have_o = false;
    uint64_t o_hash = 0;
    // shot-noise bias of the P numerator per mode (POLYBIN_FISHER_PK, POLYBIN_FISHER_PK_OPT), subtracted by the
    // estimates while present
    std::vector<double> pbias[4];
    // cross-bin partials of every alpha of one P Fisher draw (read back once a draw)
    double* dpart_all = nullptr;
    size_t dpart_all_cap = 0;
    // bispectrum shot noise: shell maps of X, Y, Z, X on the contraction grid [4][nb][cn], contraction partials and
    // output for 2 nb maps
    void* bmaps = nullptr;
    double* bpart = nullptr;
    double* bout = nullptr;
    size_t bpart_cap = 0;
};

static void uw_free(UwState* u) {
    if (!u) return;
    void* ptrs[] = {u->g2, u->xmap, u->a[0], u->a[1], u->spec[0], u->spec[1], u->spec[2], u->spec[3], u->pairs, u->qbox,
                    u->zc, u->yc, u->v1, u->v2, u->dF, u->dpart, u->dvec, u->dvec2, u->dinfo, u->dFp_inv, u->dFb_inv,
                    u->ylc, u->hbox, u->g3, u->dFl_inv, u->dFo_inv, u->bmaps, u->bpart, u->bout,
                    u->dpart_all};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    delete u;
}

void destroy_unwindowed(polybin_ctx* ctx) {
    uw_free(static_cast<UwState*>(ctx->ext));
    ctx->ext = nullptr;
}

template <typename T>
static int uw_alloc(polybin_ctx* ctx, bool need_b) {
    UwState* u = static_cast<UwState*>(ctx->ext);
    if (!u) {
        u = new (std::nothrow) UwState();
        if (!u) return fail(ctx, POLYBIN_ENOMEM, "unwindowed: out of host memory");
        ctx->ext = u;
        u->elem = sizeof(T);
    }
    const long N = ctx->ncell;
    const long nbox = (long)ctx->gx.cnt * ctx->gy.cnt * ctx->gz.cnt;
    const int nb = ctx->nb, np = nb * (nb + 1) / 2;
    auto need = [&](void** p, size_t bytes) -> int {
        if (*p) return POLYBIN_OK;
        cudaError_t e = cudaMalloc(p, bytes);
        if (e != cudaSuccess) { *p = nullptr; return fail_cuda(ctx, e, "unwindowed workspace", __FILE__, __LINE__); }
        return POLYBIN_OK;
    };
    int rc;
    if ((rc = need(&u->xmap, sizeof(T) * N))) return rc;
    if ((rc = need(&u->a[0], sizeof(T) * N))) return rc;
    if ((rc = need(&u->a[1], sizeof(T) * N))) return rc;
    for (int f = 0; f < 4; ++f)
        if ((rc = need(&u->spec[f], sizeof(C<T>) * nbox))) return rc;
    if ((rc = need(&u->g2, sizeof(T) * (size_t)nb * N))) return rc;
    if ((rc = need((void**)&u->dpart, sizeof(double) * (size_t)nb * ctx->pk_nseg * 3))) return rc;
    if ((rc = need((void**)&u->dinfo, sizeof(int)))) return rc;
    if ((rc = need((void**)&u->dvec, sizeof(double) * 4096))) return rc;
    if ((rc = need((void**)&u->dvec2, sizeof(double) * 4096))) return rc;
    if (need_b) {
        const size_t nt = ctx->Nabc.size();
        if ((rc = need(&u->pairs, sizeof(C<T>) * (size_t)4 * np * nbox))) return rc;
        if ((rc = need(&u->qbox, sizeof(C<T>) * nbox))) return rc;
        const long Mp = (std::max(ctx->nmodes, 1L) + 1) / 2 * 2;   // even row stride: 16-byte aligned rows
        const bool fresh = !u->zc;
        if ((rc = need(&u->zc, sizeof(C<T>) * nt * Mp))) return rc;
        if ((rc = need(&u->yc, sizeof(C<T>) * nt * Mp))) return rc;
        if (fresh) {   // the padding column stays zero
            PB_CUDA_OK(cudaMemset(u->zc, 0, sizeof(C<T>) * nt * Mp));
            PB_CUDA_OK(cudaMemset(u->yc, 0, sizeof(C<T>) * nt * Mp));
        }
        if ((rc = need(&u->v1, sizeof(C<T>) * (size_t)ctx->N[0] * ctx->gy.cnt * ctx->gz.cnt))) return rc;
        if ((rc = need(&u->v2, sizeof(C<T>) * (size_t)ctx->N[0] * ctx->N[1] * ctx->gz.cnt))) return rc;
    }
    return POLYBIN_OK;
}

static unsigned grid1d(long n) { return (unsigned)std::min<long>((n + 255) / 256, 152L * 16); }

// Inverse transform of a box spectrum to a real map: x-pass, y-pass, z-pass (C2R) with the 1/N of the IFT,
// and an optional pointwise multiplier on output.
template <typename T>
int run_inverse_box(polybin_ctx* ctx, const C<T>* box, C<T>* v1, C<T>* v2, T* out, const T* mulout) {
    const int N0 = ctx->N[0], N1 = ctx->N[1], N2 = ctx->N[2];
    const int By = ctx->gy.cnt, Bz = ctx->gz.cnt;
    const C<T>* tw0 = (const C<T>*)(sizeof(T) == 4 ? ctx->d_tw_f[0] : ctx->d_tw_d[0]);
    const C<T>* tw1 = (const C<T>*)(sizeof(T) == 4 ? ctx->d_tw_f[1] : ctx->d_tw_d[1]);
    const C<T>* tw2 = (const C<T>*)(sizeof(T) == 4 ? ctx->d_tw_f[2] : ctx->d_tw_d[2]);
    cudaError_t e = cudaSuccess;
    {
        const int tk = cols_per_cta_of<T>(N0);
        const size_t sm = (2 * (size_t)N0 * tk + N0) * sizeof(C<T>);
        ColBatch b;
        ColItem& it = b.it[0];
        const int ncols = By * Bz;
        it.in = box; it.out = v1;
        it.in_os = 0; it.in_es = ncols; it.out_os = 0; it.out_es = ncols;
        it.ncols = ncols; it.nouter = 1; it.rng = ctx->gx;
        PB_WITH_NT(N0, NT, {
            e = cudaFuncSetAttribute((const void*)k_col<T, +1, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
            if (e != cudaSuccess) return fail_cuda(ctx, e, "attr", __FILE__, __LINE__);
            k_col<T, +1, NT><<<dim3((ncols + tk - 1) / tk, 1, 1), 256, sm, ctx->stream>>>(b, ctx->plan[0], tw0, tk);
        })
        ctx->launches++;
    }
    {
        const int tk = cols_per_cta_of<T>(N1);
        const size_t sm = (2 * (size_t)N1 * tk + N1) * sizeof(C<T>);
        ColBatch b;
        ColItem& it = b.it[0];
        it.in = v1; it.out = v2;
        it.in_os = (long)By * Bz; it.in_es = Bz; it.out_os = (long)N1 * Bz; it.out_es = Bz;
        it.ncols = Bz; it.nouter = N0; it.rng = ctx->gy;
        PB_WITH_NT(N1, NT, {
            e = cudaFuncSetAttribute((const void*)k_col<T, +1, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
            if (e != cudaSuccess) return fail_cuda(ctx, e, "attr", __FILE__, __LINE__);
            k_col<T, +1, NT><<<dim3((Bz + tk - 1) / tk, N0, 1), 256, sm, ctx->stream>>>(b, ctx->plan[1], tw1, tk);
        })
        ctx->launches++;
    }
    {
        const int lp = lines_per_cta_of<T>(N2);
        const size_t sm = (2 * (size_t)N2 * (lp + 1) + N2) * sizeof(C<T>);
        ZInvBatch b;
        b.it[0].in = v2; b.it[0].out = out; b.it[0].kin = Bz;
        const long nlines = (long)N0 * N1;
        if (N2 == 256) {
            const int lpc = 16;
            k_inv_z256<T><<<dim3((unsigned)(((nlines + 1) / 2 + lpc - 1) / lpc), 1, 1), 256, 0, ctx->stream>>>(
                b, nlines, T(1.0 / (double)ctx->ncell), mulout, tw2, lpc);
        } else if (N2 == 512) {
            const int lpc = 16;
            k_inv_z512<T><<<dim3((unsigned)(((nlines + 1) / 2 + lpc - 1) / lpc), 1, 1), 256, 0, ctx->stream>>>(
                b, nlines, T(1.0 / (double)ctx->ncell), mulout, tw2, lpc);
        } else {
            PB_WITH_NT(N2, NT, {
                e = cudaFuncSetAttribute((const void*)k_inv_z<T, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
                if (e != cudaSuccess) return fail_cuda(ctx, e, "attr", __FILE__, __LINE__);
                k_inv_z<T, NT><<<dim3((unsigned)((nlines + 2 * lp - 1) / (2 * lp)), 1, 1), 256, sm, ctx->stream>>>(
                    b, nlines, T(1.0 / (double)ctx->ncell), mulout, ctx->plan[2], tw2, lp);
            })
        }
        ctx->launches++;
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail_cuda(ctx, e, "run_inverse_box", __FILE__, __LINE__);
    return POLYBIN_OK;
}

// Binned cross products (host result [nell][nb]) of two box spectra.
template <typename T>
static int run_cross_bin(polybin_ctx* ctx, const C<T>* X, const C<T>* A, double* dpart, std::vector<double>& out) {
    const int nb = ctx->nb, nell = ctx->nell;
    uw::k_cross_bin<T><<<dim3(nb, ctx->pk_nseg, 1), 256, 0, ctx->stream>>>(X, A, ctx->d_offs, ctx->d_coef, ctx->nmodes,
                                                                            ctx->d_bin_start, nell, ctx->pk_seg_len, dpart);
    ctx->launches++;
    std::vector<double> part((size_t)nb * ctx->pk_nseg * nell);
    PB_CUDA_OK(cudaGetLastError());
    PB_CUDA_OK(cudaMemcpyAsync(part.data(), dpart, part.size() * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    PB_CUDA_OK(cudaStreamSynchronize(ctx->stream));
    out.assign((size_t)nell * nb, 0.0);
    for (int b = 0; b < nb; ++b)
        for (int s = 0; s < ctx->pk_nseg; ++s)
            for (int l = 0; l < nell; ++l) out[(size_t)l * nb + b] += part[((size_t)b * ctx->pk_nseg + s) * nell + l];
    return POLYBIN_OK;
}

// ---------------------------------------------------------------------------------------------- P Fisher

// The binned cross products of alpha's spectrum X with A into slot alpha of dpart_all (no read-back).
template <typename T>
static int launch_cross_bin(polybin_ctx* ctx, const C<T>* X, const C<T>* A, int alpha) {
    UwState* u = static_cast<UwState*>(ctx->ext);
    const int nb = ctx->nb, nell = ctx->nell;
    const size_t per = (size_t)nb * ctx->pk_nseg * nell;
    uw::k_cross_bin<T><<<dim3(nb, ctx->pk_nseg, 1), 256, 0, ctx->stream>>>(X, A, ctx->d_offs, ctx->d_coef, ctx->nmodes,
                                                                            ctx->d_bin_start, nell, ctx->pk_seg_len,
                                                                            u->dpart_all + (size_t)alpha * per);
    ctx->launches++;
    PB_CUDA_OK(cudaGetLastError());
    return POLYBIN_OK;
}

// One Monte Carlo term of the P Fisher matrix (eq. fish-from-Q, global line of sight), host [na][na], na = nell*nb:
// F[(l,b)][(l',b')] = 1/2 (1/N) sum_k conj(FT[s IFT[Theta_b L_l FT[s a]]]) Theta_b' L_l' FT[a],  s = w n.
// The cross products of all alpha go to one device buffer read back once a draw.
template <typename T>
static int pk_fisher_draw(polybin_ctx* ctx, const float* n, const float* w, unsigned long long seed, int r,
                          std::vector<double>& F) {
    UwState* u = static_cast<UwState*>(ctx->ext);
    Work& W = ctx->w;
    const long N = ctx->ncell;
    const int nb = ctx->nb, nell = ctx->nell, na = nell * nb;
    int rc;
    T* a = (T*)u->a[0];
    uw::k_draw<T><<<grid1d((N + 3) / 4), 256, 0, ctx->stream>>>(a, N, seed, (uint32_t)r, 2u);
    ctx->launches++;
    C<T>* A = (C<T>*)u->spec[0];
    C<T>* SA = (C<T>*)u->spec[1];
    if ((rc = run_forward<T, T, float>(ctx, a, (const float*)nullptr, (const float*)nullptr, (C<T>*)W.t1, (C<T>*)W.t2, A))) return rc;
    if ((rc = run_forward<T, T, float>(ctx, a, w, n, (C<T>*)W.t1, (C<T>*)W.t2, SA))) return rc;
    F.assign((size_t)na * na, 0.0);
    const size_t per = (size_t)nb * ctx->pk_nseg * nell;
    if (u->dpart_all_cap < (size_t)na * per) {
        if (u->dpart_all) cudaFree(u->dpart_all);
        u->dpart_all = nullptr;
        u->dpart_all_cap = 0;
        PB_CUDA_OK(cudaMalloc((void**)&u->dpart_all, sizeof(double) * (size_t)na * per));
        u->dpart_all_cap = (size_t)na * per;
    }
    T* q = (T*)u->g2;
    for (int il = 0; il < nell; ++il) {
        if ((rc = ensure_fine_inv<T>(ctx))) return rc;
        if ((rc = run_shells<T>(ctx, SA, (C<T>*)W.u1f, (C<T>*)W.u2f, q, 2 * il, ctx->fg))) return rc;
        for (int b = 0; b < nb; ++b) {
            C<T>* X = (C<T>*)u->spec[2];
            if ((rc = run_forward<T, T, float>(ctx, q + (size_t)b * N, w, n, (C<T>*)W.t1, (C<T>*)W.t2, X))) return rc;
            if ((rc = launch_cross_bin<T>(ctx, X, A, il * nb + b))) return rc;
        }
    }
    std::vector<double> part((size_t)na * per);
    PB_CUDA_OK(cudaMemcpyAsync(part.data(), u->dpart_all, part.size() * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    PB_CUDA_OK(cudaStreamSynchronize(ctx->stream));
    for (int alpha = 0; alpha < na; ++alpha) {
        const double* pa = part.data() + (size_t)alpha * per;
        for (int b2 = 0; b2 < nb; ++b2)
            for (int jl = 0; jl < nell; ++jl) {
                double acc = 0.0;
                for (int sg = 0; sg < ctx->pk_nseg; ++sg) acc += pa[((size_t)b2 * ctx->pk_nseg + sg) * nell + jl];
                F[(size_t)alpha * na + jl * nb + b2] = 0.5 * acc / (double)N;
            }
    }
    return POLYBIN_OK;
}

// One Monte Carlo term of the P Fisher matrix with the optimal weighting (eq. fish-from-Q, global line of sight):
// F[(l,b)][(l',b')] = 1/2 (1/N) sum_k conj(FT[P^T S^-T IFT[Theta_b L_l FT[S^-1 P a]]]) Theta_b' L_l' FT[a], with
// S^-1 P a = G(n a / n_w) and P^T S^-T u = n G(u) / n_w, each G a conjugate-gradient solve (1 + nell nb per draw).
template <typename T>
static int pk_fisher_draw_opt(polybin_ctx* ctx, const float* n, unsigned long long seed, int r, std::vector<double>& F) {
    UwState* u = static_cast<UwState*>(ctx->ext);
    Work& W = ctx->w;
    const long N = ctx->ncell;
    const int nb = ctx->nb, nell = ctx->nell, na = nell * nb;
    int rc;
    T* a = (T*)u->a[0];
    T* sa = (T*)u->a[1];
    uw::k_draw<T><<<grid1d((N + 3) / 4), 256, 0, ctx->stream>>>(a, N, seed, (uint32_t)r, 2u);
    ctx->launches++;
    C<T>* A = (C<T>*)u->spec[0];
    C<T>* SA = (C<T>*)u->spec[1];
    if ((rc = run_forward<T, T, float>(ctx, a, (const float*)nullptr, (const float*)nullptr, (C<T>*)W.t1, (C<T>*)W.t2, A))) return rc;
    if ((rc = opt_apply<T, T, T>(ctx, a, n, 1, nullptr, 0, sa))) return rc;
    if ((rc = run_forward<T, T, float>(ctx, sa, (const float*)nullptr, (const float*)nullptr, (C<T>*)W.t1, (C<T>*)W.t2, SA))) return rc;
    F.assign((size_t)na * na, 0.0);
    std::vector<double> cross;
    T* q = (T*)u->g2;
    T* xm = (T*)u->xmap;
    for (int il = 0; il < nell; ++il) {
        if ((rc = ensure_fine_inv<T>(ctx))) return rc;
        if ((rc = run_shells<T>(ctx, SA, (C<T>*)W.u1f, (C<T>*)W.u2f, q, 2 * il, ctx->fg))) return rc;
        for (int b = 0; b < nb; ++b) {
            C<T>* X = (C<T>*)u->spec[2];
            if ((rc = opt_apply<T, T, T>(ctx, q + (size_t)b * N, nullptr, 0, n, 1, xm))) return rc;
            if ((rc = run_forward<T, T, float>(ctx, xm, (const float*)nullptr, (const float*)nullptr, (C<T>*)W.t1, (C<T>*)W.t2, X)))
                return rc;
            if ((rc = run_cross_bin<T>(ctx, X, A, u->dpart, cross))) return rc;
            const int alpha = il * nb + b;
            for (int jl = 0; jl < nell; ++jl)
                for (int b2 = 0; b2 < nb; ++b2) F[(size_t)alpha * na + jl * nb + b2] = 0.5 * cross[(size_t)jl * nb + b2] / (double)N;
        }
    }
    return POLYBIN_OK;
}

// Shot-noise bias of the P numerator (first line of eq. fish-from-Q, A = I, global line of sight), averaged over
// draws r = 0..n_mc-1 of stream 3, host [nell][nb]:
//     p_bias[(l,b)] = 1/2 (1/N) sum_{k in b} L_l Re conj(FT[S^-1 N a]) FT[S^-1 a],   N = diag(n2 / V_cell),
// with S^-1 = w (which = POLYBIN_FISHER_PK) or the optimal weighting (POLYBIN_FISHER_PK_OPT; two solves per draw).
template <typename T>
static int pk_bias_t(polybin_ctx* ctx, const float* n2, const float* w, int which, int n_mc, unsigned long long seed,
                     std::vector<double>& out) {
    int rc;
    if ((rc = uw_alloc<T>(ctx, false))) return rc;
    UwState* u = static_cast<UwState*>(ctx->ext);
    Work& W = ctx->w;
    const long N = ctx->ncell;
    const int na = ctx->nell * ctx->nb;
    const double inv_vcell = (double)N / ctx->vol;
    T* a = (T*)u->a[0];
    T* sa = (T*)u->a[1];
    T* xm = (T*)u->xmap;
    C<T>* X = (C<T>*)u->spec[0];
    C<T>* Y = (C<T>*)u->spec[1];
    out.assign(na, 0.0);
    std::vector<double> cross;
    for (int r = 0; r < n_mc; ++r) {
        uw::k_draw<T><<<grid1d((N + 3) / 4), 256, 0, ctx->stream>>>(a, N, seed, (uint32_t)r, 3u);
        ctx->launches++;
        PB_CUDA_OK(cudaGetLastError());
        if (which == 0) {
            if ((rc = run_forward<T, T, float>(ctx, a, w, n2, (C<T>*)W.t1, (C<T>*)W.t2, X))) return rc;
            if ((rc = run_forward<T, T, float>(ctx, a, w, (const float*)nullptr, (C<T>*)W.t1, (C<T>*)W.t2, Y))) return rc;
        } else {
            if ((rc = opt_apply<T, T, T>(ctx, a, n2, 1, nullptr, 0, xm))) return rc;
            if ((rc = opt_apply<T, T, T>(ctx, a, nullptr, 1, nullptr, 0, sa))) return rc;
            if ((rc = run_forward<T, T, float>(ctx, xm, (const float*)nullptr, (const float*)nullptr, (C<T>*)W.t1, (C<T>*)W.t2, X)))
                return rc;
            if ((rc = run_forward<T, T, float>(ctx, sa, (const float*)nullptr, (const float*)nullptr, (C<T>*)W.t1, (C<T>*)W.t2, Y)))
                return rc;
        }
        if ((rc = run_cross_bin<T>(ctx, X, Y, u->dpart, cross))) return rc;
        for (int i = 0; i < na; ++i) out[i] += 0.5 * cross[i] / (double)N * inv_vcell;
    }
    for (int i = 0; i < na; ++i) out[i] /= (double)n_mc;
    return POLYBIN_OK;
}

// Delta beta[X, Y, Z] for every closed triplet (eq. beta-def, ell = 0): the sum over the six assignments of (X, Y, Z)
// to the bins of sum_x g_a g_b g_c, from three contractions of 2 nb maps by nb maps on the contraction grid with the
// shell maps laid out as [X][Y][Z][X]:  [X, Y] x Z,  [Z, X] x Y,  [Y, Z] x X.  Adds fac * (that) / Delta to acc.
template <typename T>
static int beta_sym_add(polybin_ctx* ctx, double fac, std::vector<double>& acc) {
    UwState* u = static_cast<UwState*>(ctx->ext);
    const int nb = ctx->nb, n2 = 2 * nb, np2 = n2 * (n2 + 1) / 2;
    const int nt = (int)ctx->Nabc.size();
    const long cn = ctx->cg.ncell;
    const T* G = (const T*)u->bmaps;
    const T* gX = G;
    const T* gY = G + (size_t)nb * cn;
    const T* gZ = G + (size_t)2 * nb * cn;
    std::vector<double> M[3];
    const T* first[3] = {gX, gZ, gY};     // [X, Y], [Z, X], [Y, Z]
    const T* third[3] = {gZ, gY, gX};
    int rc;
    for (int c = 0; c < 3; ++c) {
        if ((rc = run_contract_any<T>(ctx, first[c], n2, third[c], nb, u->bpart, u->bpart_cap, u->bout, cn))) return rc;
        M[c].resize((size_t)np2 * nb);
        PB_CUDA_OK(cudaMemcpyAsync(M[c].data(), u->bout, sizeof(double) * M[c].size(), cudaMemcpyDeviceToHost, ctx->stream));
    }
    PB_CUDA_OK(cudaStreamSynchronize(ctx->stream));
    const double rho = ctx->cg_ratio;
    for (int t = 0; t < nt; ++t) {
        const int a = ctx->trip[3 * t], b = ctx->trip[3 * t + 1], c = ctx->trip[3 * t + 2];
        const size_t p_ab = (size_t)pair_index(n2, a, nb + b), p_ba = (size_t)pair_index(n2, b, nb + a);
        double v = 0.0;
        for (int k = 0; k < 3; ++k) v += M[k][p_ab * nb + c] + M[k][p_ba * nb + c];
        const double dl = (a == b && b == c) ? 6.0 : ((a == b || b == c) ? 2.0 : 1.0);
        acc[t] += fac * rho * v / dl;
    }
    return POLYBIN_OK;
}

// Shell maps of FT[w m] into slot `slot` of the [X][Y][Z][X] layout (slot 0 is copied to slot 3).
template <typename T, typename TIN>
static int bias_shells(polybin_ctx* ctx, const TIN* m, const float* w, int slot) {
    UwState* u = static_cast<UwState*>(ctx->ext);
    Work& W = ctx->w;
    const int nb = ctx->nb;
    const long cn = ctx->cg.ncell;
    T* G = (T*)u->bmaps + (size_t)slot * nb * cn;
    int rc;
    if ((rc = run_forward<T, TIN, float>(ctx, m, w, (const float*)nullptr, (C<T>*)W.t1, (C<T>*)W.t2, (C<T>*)W.box))) return rc;
    if ((rc = run_shells<T>(ctx, (const C<T>*)W.box, (C<T>*)W.u1, (C<T>*)W.u2, G, 0, ctx->cg))) return rc;
    if (slot == 0)
        PB_CUDA_OK(cudaMemcpyAsync((T*)u->bmaps + (size_t)3 * nb * cn, G, sizeof(T) * (size_t)nb * cn,
                                   cudaMemcpyDeviceToDevice, ctx->stream));
    return POLYBIN_OK;
}

// Shot-noise bias of the B numerator (Sec. 4.3.3; FKP weighting S^-1 = w, ell = 0, global line of sight), averaged
// over the pairs r = 0..n_mc-1 of streams 4 and 5, host [nt] in the units of b_num:
//     b_bias = -1/3 <beta[w N3[a1, a2], w a1, w a2]> + 1/2 <beta[w N2 a1, w a1, w d]>,
// N3[a1, a2] = n3 a1 a2 / V_cell^2, N2 a = d2 a / V_cell.
template <typename T>
static int bk_bias_t(polybin_ctx* ctx, const float* n3, const float* d2, const float* d, const float* w, int n_mc,
                     unsigned long long seed, std::vector<double>& out) {
    int rc;
    if ((rc = ensure_triplets(ctx))) return rc;
    if ((rc = uw_alloc<T>(ctx, false))) return rc;
    UwState* u = static_cast<UwState*>(ctx->ext);
    const int nb = ctx->nb, nt = (int)ctx->Nabc.size();
    if (2 * nb > 64) return fail(ctx, POLYBIN_EINVAL, "polybin_bk_bias: at most 32 k-bins");
    const long N = ctx->ncell, cn = ctx->cg.ncell;
    if (!u->bmaps) {
        const ContractGeom G = contract_geom(2 * nb, nb, cn);
        u->bpart_cap = (size_t)G.ncb * G.npairs * G.nh;
        cudaError_t e = cudaMalloc(&u->bmaps, sizeof(T) * (size_t)4 * nb * cn);
        if (e == cudaSuccess) e = cudaMalloc((void**)&u->bpart, sizeof(double) * u->bpart_cap);
        if (e == cudaSuccess) e = cudaMalloc((void**)&u->bout, sizeof(double) * (size_t)nb * (2 * nb + 1) * nb);
        if (e != cudaSuccess) return fail_cuda(ctx, e, "bispectrum bias workspace", __FILE__, __LINE__);
    }
    if ((rc = ensure_fine_inv<T>(ctx))) return rc;
    T* a1 = (T*)u->a[0];
    T* a2 = (T*)u->a[1];
    T* xm = (T*)u->xmap;
    const T iv = T((double)N / ctx->vol);
    out.assign(nt, 0.0);
    for (int r = 0; r < n_mc; ++r) {
        uw::k_draw<T><<<grid1d((N + 3) / 4), 256, 0, ctx->stream>>>(a1, N, seed, (uint32_t)r, 4u);
        uw::k_draw<T><<<grid1d((N + 3) / 4), 256, 0, ctx->stream>>>(a2, N, seed, (uint32_t)r, 5u);
        ctx->launches += 2;
        // -1/3 beta[w n3 a1 a2 / V^2, w a1, w a2]
        uw::k_noise_map<T><<<grid1d(N), 256, 0, ctx->stream>>>(xm, a1, a2, n3, iv * iv, N);
        ctx->launches++;
        PB_CUDA_OK(cudaGetLastError());
        if ((rc = bias_shells<T, T>(ctx, xm, w, 0))) return rc;
        if ((rc = bias_shells<T, T>(ctx, a1, w, 1))) return rc;
        if ((rc = bias_shells<T, T>(ctx, a2, w, 2))) return rc;
        if ((rc = beta_sym_add<T>(ctx, -1.0 / 3.0, out))) return rc;
        // +1/2 beta[w d2 a1 / V, w a1, w d]   (slot 1 still holds w a1)
        uw::k_noise_map<T><<<grid1d(N), 256, 0, ctx->stream>>>(xm, a1, (const T*)nullptr, d2, iv, N);
        ctx->launches++;
        PB_CUDA_OK(cudaGetLastError());
        if ((rc = bias_shells<T, T>(ctx, xm, w, 0))) return rc;
        if ((rc = bias_shells<T, float>(ctx, d, w, 2))) return rc;
        if ((rc = beta_sym_add<T>(ctx, 0.5, out))) return rc;
    }
    for (int t = 0; t < nt; ++t) out[t] /= (double)n_mc;
    return POLYBIN_OK;
}

// ---------------------------------------------------------------------------------------------- local line of sight

template <typename T>
static uw::CellGeom<T> cell_geom(const polybin_ctx* ctx) {
    uw::CellGeom<T> g;
    for (int a = 0; a < 3; ++a) {
        g.N[a] = ctx->N[a];
        g.h[a] = T(ctx->L / ctx->N[a]);
        g.obs[a] = T(ctx->observer[a]);
    }
    g.half_l = T(0.5 * ctx->L);
    return g;
}

// Workspace of the local line of sight: compact harmonic sums [3][M], one box, nb data-grid maps (Fisher only).
template <typename T>
static int uw_alloc_local(polybin_ctx* ctx, bool fisher) {
    UwState* u = static_cast<UwState*>(ctx->ext);
    const long nbox = (long)ctx->gx.cnt * ctx->gy.cnt * ctx->gz.cnt;
    if (!u->ylc) PB_CUDA_OK(cudaMalloc(&u->ylc, sizeof(double2) * 3 * std::max(ctx->nmodes, 1L)));
    if (!u->hbox) PB_CUDA_OK(cudaMalloc(&u->hbox, sizeof(C<T>) * nbox));
    if (fisher && !u->g3) PB_CUDA_OK(cudaMalloc(&u->g3, sizeof(T) * (size_t)ctx->nb * ctx->ncell));
    return POLYBIN_OK;
}

// u->ylc[l] = sum_m Ybar_lm(k) FT[Ybar_lm v](k) on the binned modes, l = 0 .. lmax/2 (l = 0: FT[v]), for the field
// v = in m1 m2 (multipliers optional); ubox receives FT[v] (the asymmetric derivative of Sec. 3.3.2 before Theta_b).
template <typename T, typename TIN>
static int local_asym(polybin_ctx* ctx, const TIN* in, const float* m1, const float* m2, C<T>* ubox) {
    UwState* u = static_cast<UwState*>(ctx->ext);
    Work& W = ctx->w;
    const long M = ctx->nmodes, N = ctx->ncell;
    const uw::CellGeom<T> cg = cell_geom<T>(ctx);
    int rc;
    if ((rc = run_forward<T, TIN, float>(ctx, in, m1, m2, (C<T>*)W.t1, (C<T>*)W.t2, ubox))) return rc;
    uw::k_ylm_gather<T><<<grid1d(M), 256, 0, ctx->stream>>>(ubox, ctx->d_offs, M, 0, 0, 1, ctx->gx, ctx->gy, ctx->gz,
                                                            u->ylc);
    ctx->launches++;
    C<T>* tmp = (C<T>*)u->spec[2];
    for (int il = 1; il < ctx->nell; ++il) {
        const int ell = 2 * il;
        for (int m = -ell; m <= ell; ++m) {
            uw::k_mul_ylm<T, TIN, float><<<grid1d(N), 256, 0, ctx->stream>>>(in, m1, m2, (T*)u->xmap, ell, m, cg);
            ctx->launches++;
            if ((rc = run_forward<T, T, float>(ctx, (const T*)u->xmap, (const float*)nullptr, (const float*)nullptr,
                                               (C<T>*)W.t1, (C<T>*)W.t2, tmp)))
                return rc;
            uw::k_ylm_gather<T><<<grid1d(M), 256, 0, ctx->stream>>>(tmp, ctx->d_offs, M, ell, m, m == -ell ? 1 : 0,
                                                                    ctx->gx, ctx->gy, ctx->gz, u->ylc + (size_t)il * M);
            ctx->launches++;
        }
    }
    PB_CUDA_OK(cudaGetLastError());
    return POLYBIN_OK;
}

// out[l][b] = sum_{k in b} w_k Re(conj(X(k)) ylc[l](k)) over the full k-grid (host result).
template <typename T>
static int run_cross_local(polybin_ctx* ctx, const C<T>* X, std::vector<double>& out) {
    UwState* u = static_cast<UwState*>(ctx->ext);
    const int nb = ctx->nb, nell = ctx->nell;
    uw::k_cross_bin_local<T><<<dim3(nb, ctx->pk_nseg, 1), 256, 0, ctx->stream>>>(
        X, u->ylc, ctx->d_offs, ctx->d_coef, ctx->nmodes, ctx->d_bin_start, nell, ctx->pk_seg_len, u->dpart);
    ctx->launches++;
    PB_CUDA_OK(cudaGetLastError());
    std::vector<double> part((size_t)nb * ctx->pk_nseg * nell);
    PB_CUDA_OK(cudaMemcpyAsync(part.data(), u->dpart, part.size() * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    PB_CUDA_OK(cudaStreamSynchronize(ctx->stream));
    out.assign((size_t)nell * nb, 0.0);
    for (int b = 0; b < nb; ++b)
        for (int sg = 0; sg < ctx->pk_nseg; ++sg)
            for (int l = 0; l < nell; ++l) out[(size_t)l * nb + b] += part[((size_t)b * ctx->pk_nseg + sg) * nell + l];
    return POLYBIN_OK;
}

// Numerator with a local line of sight (Sec. 3.3.1, eq. pk-num-fft), pixel units:
// p_num(l, b) = 1/2 (1/N) sum_{k in b} sum_m Ybar_lm(k) Re(conj(FT[Ybar_lm u]) FT[u]),  u = w d.
template <typename T>
static int pk_numerator_local_t(polybin_ctx* ctx, const float* d, const float* w, std::vector<double>& pnum) {
    UwState* u = static_cast<UwState*>(ctx->ext);
    int rc;
    C<T>* U = (C<T>*)u->spec[0];
    if ((rc = local_asym<T, float>(ctx, d, w, (const float*)nullptr, U))) return rc;
    std::vector<double> num;
    if ((rc = run_cross_local<T>(ctx, U, num))) return rc;
    pnum.resize(num.size());
    for (size_t i = 0; i < num.size(); ++i) pnum[i] = 0.5 * num[i] / (double)ctx->ncell;
    return POLYBIN_OK;
}

// One Monte Carlo term of the P Fisher matrix with a local line of sight (Sec. 3.3.2, eqs. Q-alpha-local,
// fish-from-Q; A = I), pixel units, host [na][na]:
//   F[(l,b)][(l',b')] = 1/2 (1/N) Re sum_{k in b'} conj(FT[s Q_(l,b)[s a]]) sum_m Ybar_l'm(k) FT[Ybar_l'm a](k),
//   Q_(l,b)[v] = 1/2 sum_m { Ybar_lm(x) IFT[Theta_b Ybar_lm FT[v]] + IFT[Theta_b Ybar_lm FT[Ybar_lm v]] },  s = w n
// (for l = 0 both terms are IFT[Theta_b FT[v]]).  The second terms are summed over m in k-space (one set of inverse
// transforms per l); the first take one set a harmonic, multiplied by Ybar_lm(x) and accumulated.
template <typename T>
static int pk_fisher_draw_local(polybin_ctx* ctx, const float* n, const float* w, unsigned long long seed, int r,
                                std::vector<double>& F) {
    UwState* u = static_cast<UwState*>(ctx->ext);
    Work& W = ctx->w;
    const long N = ctx->ncell;
    const int nb = ctx->nb, nell = ctx->nell, na = nell * nb;
    const uw::CellGeom<T> cg = cell_geom<T>(ctx);
    int rc;
    if ((rc = ensure_fine_inv<T>(ctx))) return rc;
    T* a = (T*)u->a[0];
    uw::k_draw<T><<<grid1d((N + 3) / 4), 256, 0, ctx->stream>>>(a, N, seed, (uint32_t)r, 2u);
    ctx->launches++;
    // asymmetric side: ylc[l'] from a
    if ((rc = local_asym<T, T>(ctx, (const T*)a, (const float*)nullptr, (const float*)nullptr, (C<T>*)u->spec[0])))
        return rc;
    // SA = FT[s a]
    C<T>* SA = (C<T>*)u->spec[1];
    if ((rc = run_forward<T, T, float>(ctx, a, w, n, (C<T>*)W.t1, (C<T>*)W.t2, SA))) return rc;
    F.assign((size_t)na * na, 0.0);
    T* Q = (T*)u->g2;
    T* q = (T*)u->g3;
    C<T>* H = (C<T>*)u->hbox;
    C<T>* X = (C<T>*)u->spec[3];
    std::vector<double> cross;
    for (int il = 0; il < nell; ++il) {
        const int ell = 2 * il;
        double fac = 1.0;
        if (ell == 0) {
            if ((rc = run_shells<T>(ctx, SA, (C<T>*)W.u1f, (C<T>*)W.u2f, Q, 0, ctx->fg))) return rc;
        } else {
            fac = 0.5;
            for (int m = -ell; m <= ell; ++m) {
                uw::k_mul_ylm<T, T, float><<<grid1d(N), 256, 0, ctx->stream>>>(a, w, n, (T*)u->xmap, ell, m, cg);
                ctx->launches++;
                if ((rc = run_forward<T, T, float>(ctx, (const T*)u->xmap, (const float*)nullptr, (const float*)nullptr,
                                                   (C<T>*)W.t1, (C<T>*)W.t2, (C<T>*)u->spec[2])))
                    return rc;
                uw::k_ylm_box_accum<T><<<grid1d((long)ctx->gx.cnt * ctx->gy.cnt * ctx->gz.cnt), 256, 0, ctx->stream>>>(
                    (const C<T>*)u->spec[2], H, ell, m, m == -ell ? 1 : 0, ctx->gx, ctx->gy, ctx->gz);
                ctx->launches++;
            }
            if ((rc = run_shells<T>(ctx, H, (C<T>*)W.u1f, (C<T>*)W.u2f, Q, 0, ctx->fg))) return rc;
            for (int m = -ell; m <= ell; ++m) {
                if ((rc = run_shells_m<T>(ctx, SA, (C<T>*)W.u1f, (C<T>*)W.u2f, q, ell, m, ctx->fg))) return rc;
                uw::k_ylm_axpy<T><<<grid1d(N), 256, 0, ctx->stream>>>(Q, q, nb, ell, m, T(1), cg);
                ctx->launches++;
            }
        }
        for (int b = 0; b < nb; ++b) {
            if ((rc = run_forward<T, T, float>(ctx, Q + (size_t)b * N, w, n, (C<T>*)W.t1, (C<T>*)W.t2, X))) return rc;
            if ((rc = run_cross_local<T>(ctx, X, cross))) return rc;
            const int alpha = il * nb + b;
            for (int jl = 0; jl < nell; ++jl)
                for (int b2 = 0; b2 < nb; ++b2)
                    F[(size_t)alpha * na + jl * nb + b2] = 0.5 * fac * cross[(size_t)jl * nb + b2] / (double)N;
        }
    }
    PB_CUDA_OK(cudaGetLastError());
    return POLYBIN_OK;
}

// ---------------------------------------------------------------------------------------------- B Fisher

// Pair spectra P_xy(k) = FT[g_x g_y](k) (x <= y, lexicographic) on the box |n_i| <= m, of the shell maps of one box
// spectrum.  The product g_x g_y has wave numbers |n_i| <= 2m, so for |k_i| <= m its transform on the contraction grid
// (more than 3m points per axis: no alias reaches the box) is (N' / N) times the data-grid one: the maps and their
// products are formed on the contraction grid and the caller multiplies the spectra by cg_ratio = N / N'.
template <typename T>
static int pair_spectra(polybin_ctx* ctx, const C<T>* U, C<T>* out) {
    UwState* u = static_cast<UwState*>(ctx->ext);
    Work& W = ctx->w;
    const long Nc = ctx->cg.ncell;
    const long nbox = (long)ctx->gx.cnt * ctx->gy.cnt * ctx->gz.cnt;
    const int nb = ctx->nb;
    int rc;
    T* g = (T*)u->g2;
    if ((rc = run_shells<T>(ctx, U, (C<T>*)W.u1, (C<T>*)W.u2, g, 0, ctx->cg))) return rc;
    int p = 0;
    for (int x = 0; x < nb; ++x)
        for (int y = x; y < nb; ++y, ++p)
            if ((rc = run_forward<T, T, T>(ctx, g + (size_t)x * Nc, g + (size_t)y * Nc, (const T*)nullptr, (C<T>*)W.t1,
                                           (C<T>*)W.t2, out + (size_t)p * nbox, ctx->cg)))
                return rc;
    return POLYBIN_OK;
}

// One Monte Carlo term of the B Fisher matrix (eq. bk-fish-def, A = I), device accumulate into u->dF [nt][nt]:
//   F_ab += (1/24) sum_x (Q_a[s a1] - Q_a[s a2]) s (Q_b[a1] - Q_b[a2]) = (1/24)(1/N) sum_k conj(Z_a) Y_b,
// Z_a = FT[s IFT[Qt_a(s a1) - Qt_a(s a2)]], Y_b = Qt_b(a1) - Qt_b(a2), Qt from eq. Q-bis-global in k-space.
template <typename T>
static int bk_fisher_draw(polybin_ctx* ctx, const float* n, const float* w, unsigned long long seed, int r) {
    UwState* u = static_cast<UwState*>(ctx->ext);
    Work& W = ctx->w;
    const long N = ctx->ncell;
    const long nbox = (long)ctx->gx.cnt * ctx->gy.cnt * ctx->gz.cnt;
    const int nb = ctx->nb, np = nb * (nb + 1) / 2;
    const int nt = (int)ctx->Nabc.size();
    const long M = ctx->nmodes;
    const long Mp = (std::max(M, 1L) + 1) / 2 * 2;   // row stride of the compact arrays
    // the split mode takes the Gram on the tensor cores from weighted Z rows; the others weight inside k_gram
    const bool tc_gram = ctx->prec == POLYBIN_SPLIT_TF32X3 && sizeof(T) == 4;
    int rc;
    T* a1 = (T*)u->a[0];
    T* a2 = (T*)u->a[1];
    uw::k_draw<T><<<grid1d((N + 3) / 4), 256, 0, ctx->stream>>>(a1, N, seed, (uint32_t)r, 0u);
    uw::k_draw<T><<<grid1d((N + 3) / 4), 256, 0, ctx->stream>>>(a2, N, seed, (uint32_t)r, 1u);
    ctx->launches += 2;
    // fields: 0 = s a1, 1 = s a2, 2 = a1, 3 = a2
    const T* src[4] = {a1, a2, a1, a2};
    C<T>* pairs = (C<T>*)u->pairs;
    for (int f = 0; f < 4; ++f) {
        const float* m1 = f < 2 ? w : nullptr;
        const float* m2 = f < 2 ? n : nullptr;
        if ((rc = run_forward<T, T, float>(ctx, src[f], m1, m2, (C<T>*)W.t1, (C<T>*)W.t2, (C<T>*)u->spec[f]))) return rc;
        if ((rc = pair_spectra<T>(ctx, (const C<T>*)u->spec[f], pairs + (size_t)f * np * nbox))) return rc;
    }
    C<T>* Zc = (C<T>*)u->zc;
    C<T>* Yc = (C<T>*)u->yc;
    C<T>* q = (C<T>*)u->qbox;
    for (int t = 0; t < nt; ++t) {
        const int a = ctx->trip[3 * t], b = ctx->trip[3 * t + 1], c = ctx->trip[3 * t + 2];
        const double dl = (a == b && b == c) ? 6.0 : ((a == b || b == c) ? 2.0 : 1.0);
        const long pab = (long)pair_index(nb, a, b) * nbox, pbc = (long)pair_index(nb, b, c) * nbox,
                   pac = (long)pair_index(nb, a, c) * nbox;
        // Y_b: fields a1, a2 (compact binned modes)
        uw::k_qcomb<T><<<grid1d(nbox), 256, 0, ctx->stream>>>(pairs + (size_t)2 * np * nbox, pairs + (size_t)3 * np * nbox,
                                                              pab, pbc, pac, a, b, c, T(2.0 / dl * ctx->cg_ratio),
                                                              ctx->gx, ctx->gy, ctx->gz, ctx->d_lut, ctx->smax, q);
        uw::k_gather<T><<<grid1d(M), 256, 0, ctx->stream>>>(q, ctx->d_offs, M, Yc + (size_t)t * Mp);
        // Z_a: fields s a1, s a2 -> real map -> times s -> forward -> compact
        uw::k_qcomb<T><<<grid1d(nbox), 256, 0, ctx->stream>>>(pairs, pairs + (size_t)np * nbox, pab, pbc, pac, a, b, c,
                                                              T(2.0 / dl * ctx->cg_ratio), ctx->gx, ctx->gy, ctx->gz,
                                                              ctx->d_lut, ctx->smax, q);
        ctx->launches += 3;
        if ((rc = run_inverse_box<T>(ctx, q, (C<T>*)u->v1, (C<T>*)u->v2, (T*)u->xmap, (const T*)nullptr))) return rc;
        if ((rc = run_forward<T, T, float>(ctx, (const T*)u->xmap, w, n, (C<T>*)W.t1, (C<T>*)W.t2, q))) return rc;
        uw::k_gather<T><<<grid1d(M), 256, 0, ctx->stream>>>(q, ctx->d_offs, M, Zc + (size_t)t * Mp,
                                                            tc_gram ? ctx->d_coef : nullptr);
        ctx->launches++;
    }
    if (tc_gram) {
        // F += (1/24)(1/N) Re sum_m w_m conj(Z_a) Y_b as a real Gram over interleaved (re, im): K = 2 Mp
        PB_CUDA_OK(cudaGetLastError());
        return run_gram_tc(ctx, (const float*)Zc, nt, (const float*)Yc, nt, 2 * Mp, 1.0 / (24.0 * (double)N), u->dF);
    }
    dim3 g((nt + 31) / 32, (nt + 31) / 32, 1);
    uw::k_gram<T><<<g, 256, 0, ctx->stream>>>(Zc, Yc, ctx->d_coef, nt, nt, M, Mp, 1.0 / (24.0 * (double)N), u->dF);
    ctx->launches++;
    PB_CUDA_OK(cudaGetLastError());
    return POLYBIN_OK;
}

// ---------------------------------------------------------------------------------------------- solve

// X = A^-1 B in FP64 on the device (A n x n, B n x nrhs, host row major); optionally also A^-1.
static int gpu_solve(polybin_ctx* ctx, const double* A, int n, const double* B, int nrhs, double* X) {
    double *dA = nullptr, *dB = nullptr;
    int* dinfo = nullptr;
    int rc = POLYBIN_OK;
    cudaError_t e = cudaMalloc(&dA, sizeof(double) * (size_t)n * n);
    if (e == cudaSuccess) e = cudaMalloc(&dB, sizeof(double) * (size_t)n * nrhs);
    if (e == cudaSuccess) e = cudaMalloc(&dinfo, sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpyAsync(dA, A, sizeof(double) * (size_t)n * n, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dB, B, sizeof(double) * (size_t)n * nrhs, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) {
        uw::k_lu_solve<<<1, 1024, 0, ctx->stream>>>(dA, n, dB, nrhs, dinfo);
        ctx->launches++;
        e = cudaGetLastError();
    }
    int info = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(X, dB, sizeof(double) * (size_t)n * nrhs, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&info, dinfo, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) rc = fail_cuda(ctx, e, "gpu_solve", __FILE__, __LINE__);
    else if (info) rc = fail(ctx, POLYBIN_EINVAL, "solve: matrix is singular (zero pivot in column %d)", info - 1);
    if (dA) cudaFree(dA);
    if (dB) cudaFree(dB);
    if (dinfo) cudaFree(dinfo);
    return rc;
}

// ---------------------------------------------------------------------------------------------- checkpoint

static uint64_t fnv1a(const void* p, size_t n, uint64_t h = 1469598103934665603ULL) {
    const unsigned char* c = static_cast<const unsigned char*>(p);
    for (size_t i = 0; i < n; ++i) { h ^= c[i]; h *= 1099511628211ULL; }
    return h;
}

struct CkptHeader {
    char magic[8];
    int32_t which, nalpha;
    int64_t done;
    uint64_t seed, setup_hash, mask_hash;
};

static uint64_t setup_hash(const polybin_ctx* ctx, int which) {
    uint64_t h = fnv1a(ctx->N, sizeof(ctx->N));
    h = fnv1a(ctx->edges.data(), sizeof(double) * ctx->edges.size(), h);
    h = fnv1a(&ctx->L, sizeof(ctx->L), h);
    h = fnv1a(&ctx->lmax, sizeof(ctx->lmax), h);
    h = fnv1a(&which, sizeof(which), h);
    h = fnv1a(&ctx->prec, sizeof(ctx->prec), h);
    if (which == 2) h = fnv1a(ctx->observer, sizeof(ctx->observer), h);
    if (which == 3) {
        const uint64_t o = opt_hash(ctx);
        h = fnv1a(&o, sizeof(o), h);
    }
    return h;
}

static int mask_hash(polybin_ctx* ctx, const float* n, const float* w, uint64_t* out) {
    std::vector<float> hn(ctx->ncell), hw(w ? ctx->ncell : 0);
    PB_CUDA_OK(cudaMemcpyAsync(hn.data(), n, sizeof(float) * ctx->ncell, cudaMemcpyDeviceToHost, ctx->stream));
    if (w) PB_CUDA_OK(cudaMemcpyAsync(hw.data(), w, sizeof(float) * ctx->ncell, cudaMemcpyDeviceToHost, ctx->stream));
    PB_CUDA_OK(cudaStreamSynchronize(ctx->stream));
    *out = fnv1a(hw.data(), sizeof(float) * hw.size(), fnv1a(hn.data(), sizeof(float) * hn.size()));
    return POLYBIN_OK;
}

// Returns POLYBIN_OK and fills sum/done if a matching checkpoint exists (done = 0 if there is none);
// POLYBIN_EINVAL if the file exists but is corrupted or belongs to another setup.
static int ckpt_load(polybin_ctx* ctx, const char* path, const CkptHeader& want, std::vector<double>& sum, int64_t* done) {
    *done = 0;
    FILE* f = fopen(path, "rb");
    if (!f) return POLYBIN_OK;
    CkptHeader h;
    const size_t na2 = (size_t)want.nalpha * want.nalpha;
    std::vector<double> data(na2);
    uint64_t check = 0;
    const bool ok = fread(&h, sizeof(h), 1, f) == 1 && fread(data.data(), sizeof(double), na2, f) == na2 &&
                    fread(&check, sizeof(check), 1, f) == 1;
    fclose(f);
    if (!ok || memcmp(h.magic, "PBFISH01", 8) != 0 || check != fnv1a(data.data(), sizeof(double) * na2, fnv1a(&h, sizeof(h))))
        return fail(ctx, POLYBIN_EINVAL, "checkpoint %s is corrupted", path);
    if (h.which != want.which || h.nalpha != want.nalpha || h.seed != want.seed || h.setup_hash != want.setup_hash ||
        h.mask_hash != want.mask_hash)
        return fail(ctx, POLYBIN_EINVAL, "checkpoint %s belongs to a different setup (bins, mask, seed or mode)", path);
    sum = data;
    *done = h.done;
    return POLYBIN_OK;
}

static int ckpt_save(polybin_ctx* ctx, const char* path, CkptHeader h, const std::vector<double>& sum) {
    std::string tmp = std::string(path) + ".tmp";
    FILE* f = fopen(tmp.c_str(), "wb");
    if (!f) return fail(ctx, POLYBIN_EINVAL, "cannot write checkpoint %s", tmp.c_str());
    const uint64_t check = fnv1a(sum.data(), sizeof(double) * sum.size(), fnv1a(&h, sizeof(h)));
    const bool ok = fwrite(&h, sizeof(h), 1, f) == 1 && fwrite(sum.data(), sizeof(double), sum.size(), f) == sum.size() &&
                    fwrite(&check, sizeof(check), 1, f) == 1;
    fclose(f);
    if (!ok || rename(tmp.c_str(), path) != 0) return fail(ctx, POLYBIN_EINVAL, "cannot write checkpoint %s", path);
    return POLYBIN_OK;
}

// ---------------------------------------------------------------------------------------------- drivers

template <typename T>
static int fisher_sum(polybin_ctx* ctx, const float* n, const float* w, unsigned long long seed, int which, int r0, int r1,
                      std::vector<double>& sum, double* per_draw) {
    UwState* u = static_cast<UwState*>(ctx->ext);
    int rc;
    const int na = which != 1 ? ctx->nell * ctx->nb : (int)ctx->Nabc.size();
    if (sum.size() != (size_t)na * na) sum.assign((size_t)na * na, 0.0);
    std::vector<double> F;
    for (int r = r0; r < r1; ++r) {
        if (which == 0) {
            if ((rc = pk_fisher_draw<T>(ctx, n, w, seed, r, F))) return rc;
        } else if (which == 2) {
            if ((rc = pk_fisher_draw_local<T>(ctx, n, w, seed, r, F))) return rc;
        } else if (which == 3) {
            if ((rc = pk_fisher_draw_opt<T>(ctx, n, seed, r, F))) return rc;
        } else {
            if (!u->dF) {
                cudaError_t e = cudaMalloc(&u->dF, sizeof(double) * (size_t)na * na);
                if (e != cudaSuccess) return fail_cuda(ctx, e, "cudaMalloc Fisher", __FILE__, __LINE__);
            }
            PB_CUDA_OK(cudaMemsetAsync(u->dF, 0, sizeof(double) * (size_t)na * na, ctx->stream));
            if ((rc = bk_fisher_draw<T>(ctx, n, w, seed, r))) return rc;
            F.resize((size_t)na * na);
            PB_CUDA_OK(cudaMemcpyAsync(F.data(), u->dF, sizeof(double) * F.size(), cudaMemcpyDeviceToHost, ctx->stream));
            PB_CUDA_OK(cudaStreamSynchronize(ctx->stream));
        }
        for (size_t i = 0; i < F.size(); ++i) sum[i] += F[i];
        if (per_draw) std::memcpy(per_draw + (size_t)(r - r0) * na * na, F.data(), sizeof(double) * F.size());
    }
    return POLYBIN_OK;
}

// Caches F and F^-1 (host copies, F^-1 on the device) of mode `which` in the context.
static int store_fisher(polybin_ctx* ctx, int which, const std::vector<double>& F, const std::vector<double>& Finv) {
    UwState* u = static_cast<UwState*>(ctx->ext);
    const size_t na2 = F.size();
    double** dinv = which == 0 ? &u->dFp_inv : (which == 1 ? &u->dFb_inv : (which == 2 ? &u->dFl_inv : &u->dFo_inv));
    if (!*dinv) {
        cudaError_t e = cudaMalloc(dinv, sizeof(double) * na2);
        if (e != cudaSuccess) return fail_cuda(ctx, e, "cudaMalloc Finv", __FILE__, __LINE__);
    }
    PB_CUDA_OK(cudaMemcpyAsync(*dinv, Finv.data(), sizeof(double) * na2, cudaMemcpyHostToDevice, ctx->stream));
    PB_CUDA_OK(cudaStreamSynchronize(ctx->stream));
    if (which == 0) { u->Fp = F; u->Fp_inv = Finv; u->have_p = true; }
    else if (which == 1) { u->Fb = F; u->Fb_inv = Finv; u->have_b = true; }
    else if (which == 2) { u->Fl = F; u->Fl_inv = Finv; u->have_l = true; }
    else { u->Fo = F; u->Fo_inv = Finv; u->have_o = true; u->o_hash = opt_hash(ctx); }
    return POLYBIN_OK;
}

template <typename T>
static int fisher_t(polybin_ctx* ctx, const float* n, const float* w, int n_mc, unsigned long long seed, int which,
                    double* fisher_out, double* fisher_inv_out, const char* ckpt) {
    int rc;
    if (which == 1 && (rc = ensure_triplets(ctx))) return rc;
    if ((rc = uw_alloc<T>(ctx, which == 1))) return rc;
    if (which == 2 && (rc = uw_alloc_local<T>(ctx, true))) return rc;
    if (which == 3 && !opt_hash(ctx))
        return fail(ctx, POLYBIN_ENOTREADY, "polybin_fisher(POLYBIN_FISHER_PK_OPT): call polybin_set_optimal first");
    const int na = which != 1 ? ctx->nell * ctx->nb : (int)ctx->Nabc.size();
    std::vector<double> sum((size_t)na * na, 0.0);
    int64_t done = 0;
    CkptHeader h;
    memcpy(h.magic, "PBFISH01", 8);
    h.which = which; h.nalpha = na; h.done = 0; h.seed = seed; h.setup_hash = setup_hash(ctx, which); h.mask_hash = 0;
    if (ckpt) {
        if ((rc = mask_hash(ctx, n, w, &h.mask_hash))) return rc;
        if ((rc = ckpt_load(ctx, ckpt, h, sum, &done))) return rc;
        if (done > n_mc) return fail(ctx, POLYBIN_EINVAL, "checkpoint holds %lld draws, more than n_mc = %d", (long long)done, n_mc);
    }
    for (int r = (int)done; r < n_mc; ++r) {
        if ((rc = fisher_sum<T>(ctx, n, w, seed, which, r, r + 1, sum, nullptr))) return rc;
        if (ckpt) {
            h.done = r + 1;
            if ((rc = ckpt_save(ctx, ckpt, h, sum))) return rc;
        }
    }
    std::vector<double> F(sum.size());
    for (size_t i = 0; i < F.size(); ++i) F[i] = sum[i] / (double)n_mc;
    std::vector<double> I((size_t)na * na, 0.0), Finv((size_t)na * na);
    for (int i = 0; i < na; ++i) I[(size_t)i * na + i] = 1.0;
    if ((rc = gpu_solve(ctx, F.data(), na, I.data(), na, Finv.data()))) return rc;
    if (fisher_out) std::memcpy(fisher_out, F.data(), sizeof(double) * F.size());
    if (fisher_inv_out) std::memcpy(fisher_inv_out, Finv.data(), sizeof(double) * Finv.size());
    return store_fisher(ctx, which, F, Finv);
}

// x = F^-1 v on the device (FP64).
static int apply_inverse(polybin_ctx* ctx, const double* dinv, int na, const std::vector<double>& v, std::vector<double>& x) {
    UwState* u = static_cast<UwState*>(ctx->ext);
    double *dv = u->dvec, *dx = u->dvec2;
    double *tmpv = nullptr, *tmpx = nullptr;
    if (na > 4096) {
        PB_CUDA_OK(cudaMalloc(&tmpv, sizeof(double) * na));
        PB_CUDA_OK(cudaMalloc(&tmpx, sizeof(double) * na));
        dv = tmpv; dx = tmpx;
    }
    x.assign(na, 0.0);
    PB_CUDA_OK(cudaMemcpyAsync(dv, v.data(), sizeof(double) * na, cudaMemcpyHostToDevice, ctx->stream));
    uw::k_gemv<<<(na + 127) / 128, 128, 0, ctx->stream>>>(dinv, dv, na, dx);
    ctx->launches++;
    PB_CUDA_OK(cudaGetLastError());
    PB_CUDA_OK(cudaMemcpyAsync(x.data(), dx, sizeof(double) * na, cudaMemcpyDeviceToHost, ctx->stream));
    PB_CUDA_OK(cudaStreamSynchronize(ctx->stream));
    if (tmpv) cudaFree(tmpv);
    if (tmpx) cudaFree(tmpx);
    return POLYBIN_OK;
}

template <typename T>
static int pk_unwindowed_t(polybin_ctx* ctx, const float* d, const float* w, double* pk_out, double* pnum_out) {
    int rc;
    if ((rc = uw_alloc<T>(ctx, false))) return rc;
    UwState* u = static_cast<UwState*>(ctx->ext);
    Work& W = ctx->w;
    const int nb = ctx->nb, na = ctx->nell * nb;
    if ((rc = run_forward<T, float, float>(ctx, d, w, (const float*)nullptr, (C<T>*)W.t1, (C<T>*)W.t2, (C<T>*)W.box))) return rc;
    std::vector<double> num;
    if ((rc = run_pkbin<T>(ctx, (const C<T>*)W.box, num))) return rc;
    std::vector<double> pnum(na);
    for (int i = 0; i < na; ++i) pnum[i] = 0.5 * num[i] / (double)ctx->ncell;
    if (pnum_out) std::memcpy(pnum_out, pnum.data(), sizeof(double) * na);
    if (!pk_out) return POLYBIN_OK;
    if (!u->have_p) return fail(ctx, POLYBIN_ENOTREADY, "polybin_pk_unwindowed: run polybin_fisher(POLYBIN_FISHER_PK) first");
    if (!u->pbias[0].empty())
        for (int i = 0; i < na; ++i) pnum[i] -= u->pbias[0][i];
    std::vector<double> x;
    if ((rc = apply_inverse(ctx, u->dFp_inv, na, pnum, x))) return rc;
    for (int i = 0; i < na; ++i) pk_out[i] = x[i] * ctx->vol / (double)ctx->ncell;
    return POLYBIN_OK;
}

template <typename T>
static int bk_unwindowed_t(polybin_ctx* ctx, const float* d, const float* w, const float* mocks, int n_mocks,
                           double* bk_out, double* bnum_out, double* lin_out, const double* bias = nullptr) {
    int rc;
    if ((rc = ensure_triplets(ctx))) return rc;
    if ((rc = uw_alloc<T>(ctx, false))) return rc;
    UwState* u = static_cast<UwState*>(ctx->ext);
    Work& W = ctx->w;
    const long N = ctx->ncell;
    const int nb = ctx->nb, np = nb * (nb + 1) / 2;
    const int nt = (int)ctx->Nabc.size();
    // u = w d -> g[u] (kept in W.g), on the contraction grid: every sum below is cg_ratio times its value there
    const double rho = ctx->cg_ratio;
    const long cn = ctx->cg.ncell;
    if ((rc = run_forward<T, float, float>(ctx, d, w, (const float*)nullptr, (C<T>*)W.t1, (C<T>*)W.t2, (C<T>*)W.box))) return rc;
    if ((rc = run_shells<T>(ctx, (const C<T>*)W.box, (C<T>*)W.u1, (C<T>*)W.u2, (T*)W.g, 0, ctx->cg))) return rc;
    std::vector<double> S(std::max(nt, 1), 0.0), lin(nt, 0.0), Mv((size_t)np * nb);
    if (nt > 0) {
        if ((rc = run_triplet_sums<T>(ctx, (const T*)W.g, ctx->d_S))) return rc;
        PB_CUDA_OK(cudaMemcpyAsync(S.data(), ctx->d_S, sizeof(double) * nt, cudaMemcpyDeviceToHost, ctx->stream));
        PB_CUDA_OK(cudaStreamSynchronize(ctx->stream));
        for (int t = 0; t < nt; ++t) S[t] *= rho;
    }
    for (int i = 0; i < n_mocks; ++i) {
        const float* mock = mocks + (size_t)i * N;
        if ((rc = run_forward<T, float, float>(ctx, mock, w, (const float*)nullptr, (C<T>*)W.t1, (C<T>*)W.t2, (C<T>*)W.box))) return rc;
        if ((rc = run_shells<T>(ctx, (const C<T>*)W.box, (C<T>*)W.u1, (C<T>*)W.u2, (T*)u->g2, 0, ctx->cg))) return rc;
        // M[(j<=k) over v][i over u] = sum_x g_j[v] g_k[v] g_i[u]
        if ((rc = run_contract_any<T>(ctx, (const T*)u->g2, nb, (const T*)W.g, nb, W.partial, W.partial_cap, W.mout, cn)))
            return rc;
        PB_CUDA_OK(cudaMemcpyAsync(Mv.data(), W.mout, sizeof(double) * Mv.size(), cudaMemcpyDeviceToHost, ctx->stream));
        PB_CUDA_OK(cudaStreamSynchronize(ctx->stream));
        for (int t = 0; t < nt; ++t) {
            const int a = ctx->trip[3 * t], b = ctx->trip[3 * t + 1], c = ctx->trip[3 * t + 2];
            lin[t] += rho * (Mv[(size_t)pair_index(nb, b, c) * nb + a] + Mv[(size_t)pair_index(nb, a, c) * nb + b] +
                             Mv[(size_t)pair_index(nb, a, b) * nb + c]);
        }
    }
    std::vector<double> bnum(nt);
    for (int t = 0; t < nt; ++t) {
        const int a = ctx->trip[3 * t], b = ctx->trip[3 * t + 1], c = ctx->trip[3 * t + 2];
        const double dl = (a == b && b == c) ? 6.0 : ((a == b || b == c) ? 2.0 : 1.0);
        if (n_mocks > 0) lin[t] /= n_mocks;
        bnum[t] = (S[t] - lin[t]) / dl;
    }
    if (bnum_out) std::memcpy(bnum_out, bnum.data(), sizeof(double) * nt);
    if (lin_out) std::memcpy(lin_out, lin.data(), sizeof(double) * nt);
    if (!bk_out) return POLYBIN_OK;
    if (!u->have_b) return fail(ctx, POLYBIN_ENOTREADY, "polybin_bk_unwindowed: run polybin_fisher(POLYBIN_FISHER_BK) first");
    if (bias)
        for (int t = 0; t < nt; ++t) bnum[t] -= bias[t];
    std::vector<double> x;
    if ((rc = apply_inverse(ctx, u->dFb_inv, nt, bnum, x))) return rc;
    const double v2 = (ctx->vol / (double)N) * (ctx->vol / (double)N);
    for (int t = 0; t < nt; ++t) bk_out[t] = x[t] * v2;
    return POLYBIN_OK;
}

// Ideal bispectrum multipoles with a local line of sight (Sec. 4.3.1, eq. g-ell-def with its Ybar_lm expansion):
// H_ell = sum_m Ybar_lm(k) FT[Ybar_lm(x) u] on the box (2 ell + 1 forward transforms of the harmonic-weighted field),
// g_{c,ell} = IFT[Theta_c H_ell] on the contraction grid beside the ell = 0 maps g, S^ell = sum_x g_a g_b g_{c,ell}
// and B_ell = (2 ell + 1)(V^2 / N^3) S^ell / T_abc on the device (the normalisation of the global multipoles).
template <typename T>
static int bk_multipoles_local_t(polybin_ctx* ctx, const float* delta, int batch, int lmax_b, double* bk_out) {
    int rc;
    if ((rc = ensure_triplets(ctx))) return rc;
    if ((rc = uw_alloc<T>(ctx, false))) return rc;
    if ((rc = uw_alloc_local<T>(ctx, false))) return rc;
    UwState* u = static_cast<UwState*>(ctx->ext);
    Work& w = ctx->w;
    const size_t nt = ctx->Nabc.size();
    const int nl = lmax_b / 2 + 1;
    const long N = ctx->ncell, nbox = (long)ctx->gx.cnt * ctx->gy.cnt * ctx->gz.cnt;
    if (lmax_b > 0 && !w.g2) PB_CUDA_OK(cudaMalloc(&w.g2, sizeof(T) * (size_t)ctx->nb * ctx->cg.ncell));
    const uw::CellGeom<T> geom = cell_geom<T>(ctx);
    C<T>* H = (C<T>*)u->hbox;
    C<T>* tmp = (C<T>*)u->spec[2];
    for (int f = 0; f < batch; ++f) {
        const float* in;
        if ((rc = resolve_input(ctx, delta + (size_t)f * N, N, &in))) return rc;
        if ((rc = run_forward<T, float, float>(ctx, in, (const float*)nullptr, (const float*)nullptr, (C<T>*)w.t1,
                                               (C<T>*)w.t2, (C<T>*)w.box)))
            return rc;
        if (nt == 0) continue;
        if ((rc = run_shells<T>(ctx, (const C<T>*)w.box, (C<T>*)w.u1, (C<T>*)w.u2, (T*)w.g, 0, ctx->cg))) return rc;
        for (int il = 0; il < nl; ++il) {
            const int ell = 2 * il;
            if (ell == 0) {
                if ((rc = run_triplet_sums<T>(ctx, (const T*)w.g, ctx->d_S))) return rc;
            } else {
                for (int m = -ell; m <= ell; ++m) {
                    uw::k_mul_ylm<T, float, float><<<grid1d(N), 256, 0, ctx->stream>>>(
                        in, (const float*)nullptr, (const float*)nullptr, (T*)u->xmap, ell, m, geom);
                    ctx->launches++;
                    if ((rc = run_forward<T, T, float>(ctx, (const T*)u->xmap, (const float*)nullptr,
                                                       (const float*)nullptr, (C<T>*)w.t1, (C<T>*)w.t2, tmp)))
                        return rc;
                    uw::k_ylm_box_accum<T><<<grid1d(nbox), 256, 0, ctx->stream>>>(tmp, H, ell, m, m == -ell ? 1 : 0,
                                                                                  ctx->gx, ctx->gy, ctx->gz);
                    ctx->launches++;
                }
                PB_CUDA_OK(cudaGetLastError());
                if ((rc = run_shells<T>(ctx, H, (C<T>*)w.u1, (C<T>*)w.u2, (T*)w.g2, 0, ctx->cg))) return rc;
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

template int run_inverse_box<float>(polybin_ctx*, const float2*, float2*, float2*, float*, const float*);
template int run_inverse_box<double>(polybin_ctx*, const double2*, double2*, double2*, double*, const double*);

// Unwindowed P_ell with the optimal weighting: p_num of eq. pk-num-fft with u = S^-1 d = G(d / n_w), p = F^-1 p_num
// with the Fisher matrix of the same weighting, physical units p V / N.
template <typename T>
static int pk_unwindowed_opt_t(polybin_ctx* ctx, const float* d, double* pk_out, double* pnum_out) {
    int rc;
    if ((rc = uw_alloc<T>(ctx, false))) return rc;
    UwState* u = static_cast<UwState*>(ctx->ext);
    Work& W = ctx->w;
    const int na = ctx->nell * ctx->nb;
    T* xm = (T*)u->xmap;
    if ((rc = opt_apply<T, float, T>(ctx, d, nullptr, 1, nullptr, 0, xm))) return rc;
    if ((rc = run_forward<T, T, float>(ctx, xm, (const float*)nullptr, (const float*)nullptr, (C<T>*)W.t1, (C<T>*)W.t2,
                                       (C<T>*)W.box)))
        return rc;
    std::vector<double> num;
    if ((rc = run_pkbin<T>(ctx, (const C<T>*)W.box, num))) return rc;
    std::vector<double> pnum(na);
    for (int i = 0; i < na; ++i) pnum[i] = 0.5 * num[i] / (double)ctx->ncell;
    if (pnum_out) std::memcpy(pnum_out, pnum.data(), sizeof(double) * na);
    if (!pk_out) return POLYBIN_OK;
    if (!u->have_o) return fail(ctx, POLYBIN_ENOTREADY, "polybin_pk_unwindowed_opt: run polybin_fisher(POLYBIN_FISHER_PK_OPT) first");
    if (u->o_hash != opt_hash(ctx))
        return fail(ctx, POLYBIN_ENOTREADY, "polybin_pk_unwindowed_opt: the optimal weighting changed since its Fisher matrix was computed");
    if (!u->pbias[3].empty())
        for (int i = 0; i < na; ++i) pnum[i] -= u->pbias[3][i];
    std::vector<double> x;
    if ((rc = apply_inverse(ctx, u->dFo_inv, na, pnum, x))) return rc;
    for (int i = 0; i < na; ++i) pk_out[i] = x[i] * ctx->vol / (double)ctx->ncell;
    return POLYBIN_OK;
}

}  // namespace pb

using namespace pb;

static bool is_device_ptr(const void* p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) { cudaGetLastError(); return false; }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

extern "C" int polybin_fkp_weights(polybin_ctx* ctx, const float* n_dev, double p_fkp, float* w_dev) {
    if (!ctx || !n_dev || !w_dev) return fail(ctx, POLYBIN_EINVAL, "polybin_fkp_weights: NULL argument");
    if (!is_device_ptr(n_dev) || !is_device_ptr(w_dev)) return fail(ctx, POLYBIN_EINVAL, "polybin_fkp_weights: device pointers required");
    uw::k_fkp<float><<<grid1d(ctx->ncell), 256, 0, ctx->stream>>>(n_dev, p_fkp, w_dev, ctx->ncell);
    ctx->launches++;
    PB_CUDA_OK(cudaGetLastError());
    PB_CUDA_OK(cudaStreamSynchronize(ctx->stream));
    return POLYBIN_OK;
}

extern "C" int polybin_mc_draw(polybin_ctx* ctx, unsigned long long seed, int draw, int stream, float* out_dev) {
    if (!ctx || !out_dev || draw < 0 || stream < 0) return fail(ctx, POLYBIN_EINVAL, "polybin_mc_draw: bad argument");
    uw::k_draw<float><<<grid1d((ctx->ncell + 3) / 4), 256, 0, ctx->stream>>>(out_dev, ctx->ncell, seed, (uint32_t)draw, (uint32_t)stream);
    ctx->launches++;
    PB_CUDA_OK(cudaGetLastError());
    PB_CUDA_OK(cudaStreamSynchronize(ctx->stream));
    return POLYBIN_OK;
}

static int check_uw_args(polybin_ctx* ctx, const float* a, const float* b, const char* what) {
    if (!ctx || !a || !b) return fail(ctx, POLYBIN_EINVAL, "%s: NULL argument", what);
    if (!is_device_ptr(a) || !is_device_ptr(b)) return fail(ctx, POLYBIN_EINVAL, "%s: device pointers required", what);
    return POLYBIN_OK;
}

// The optimal weighting (which = 3) takes no weight map: w may be NULL.
static int check_fisher_args(polybin_ctx* ctx, const float* n, const float* w, int which, const char* what) {
    if (which == 3 && !w) return check_uw_args(ctx, n, n, what);
    return check_uw_args(ctx, n, w, what);
}

extern "C" int polybin_fisher(polybin_ctx* ctx, const float* n_dev, const float* w_dev, int n_mc, unsigned long long seed,
                              int which, double* fisher_out, double* fisher_inv_out, const char* checkpoint_path) {
    int rc = check_fisher_args(ctx, n_dev, w_dev, which, "polybin_fisher");
    if (rc) return rc;
    if (n_mc < 1 || which < 0 || which > 3) return fail(ctx, POLYBIN_EINVAL, "polybin_fisher: n_mc >= 1, which in {0, 1, 2, 3}");
    if (which == 3) w_dev = nullptr;
    return ctx->prec == POLYBIN_FP64 ? fisher_t<double>(ctx, n_dev, w_dev, n_mc, seed, which, fisher_out, fisher_inv_out, checkpoint_path)
                                     : fisher_t<float>(ctx, n_dev, w_dev, n_mc, seed, which, fisher_out, fisher_inv_out, checkpoint_path);
}

extern "C" int polybin_fisher_draws(polybin_ctx* ctx, const float* n_dev, const float* w_dev, unsigned long long seed,
                                    int which, int draw_begin, int draw_end, double* per_draw_out) {
    int rc = check_fisher_args(ctx, n_dev, w_dev, which, "polybin_fisher_draws");
    if (rc) return rc;
    if (!per_draw_out || draw_begin < 0 || draw_end < draw_begin || which < 0 || which > 3)
        return fail(ctx, POLYBIN_EINVAL, "polybin_fisher_draws: bad argument");
    if (which == 1 && (rc = ensure_triplets(ctx))) return rc;
    if (which == 3 && !opt_hash(ctx))
        return fail(ctx, POLYBIN_ENOTREADY, "polybin_fisher_draws(POLYBIN_FISHER_PK_OPT): call polybin_set_optimal first");
    std::vector<double> sum;
    if (ctx->prec == POLYBIN_FP64) {
        if ((rc = uw_alloc<double>(ctx, which == 1))) return rc;
        if (which == 2 && (rc = uw_alloc_local<double>(ctx, true))) return rc;
        return fisher_sum<double>(ctx, n_dev, w_dev, seed, which, draw_begin, draw_end, sum, per_draw_out);
    }
    if ((rc = uw_alloc<float>(ctx, which == 1))) return rc;
    if (which == 2 && (rc = uw_alloc_local<float>(ctx, true))) return rc;
    return fisher_sum<float>(ctx, n_dev, w_dev, seed, which, draw_begin, draw_end, sum, per_draw_out);
}

extern "C" int polybin_set_fisher(polybin_ctx* ctx, int which, const double* fisher) {
    if (!ctx || !fisher || which < 0 || which > 3) return fail(ctx, POLYBIN_EINVAL, "polybin_set_fisher: bad argument");
    if (which == 3 && !opt_hash(ctx))
        return fail(ctx, POLYBIN_ENOTREADY, "polybin_set_fisher(POLYBIN_FISHER_PK_OPT): call polybin_set_optimal first");
    int rc;
    if (which == 1 && (rc = ensure_triplets(ctx))) return rc;
    if ((rc = ctx->prec == POLYBIN_FP64 ? uw_alloc<double>(ctx, false) : uw_alloc<float>(ctx, false))) return rc;
    const int na = which != 1 ? ctx->nell * ctx->nb : (int)ctx->Nabc.size();
    std::vector<double> F(fisher, fisher + (size_t)na * na), I((size_t)na * na, 0.0), Finv((size_t)na * na);
    for (int i = 0; i < na; ++i) I[(size_t)i * na + i] = 1.0;
    if ((rc = gpu_solve(ctx, F.data(), na, I.data(), na, Finv.data()))) return rc;
    return store_fisher(ctx, which, F, Finv);
}

extern "C" int polybin_set_observer(polybin_ctx* ctx, const double pos[3]) {
    if (!ctx || !pos) return fail(ctx, POLYBIN_EINVAL, "polybin_set_observer: NULL argument");
    for (int a = 0; a < 3; ++a)
        if (!std::isfinite(pos[a])) return fail(ctx, POLYBIN_EINVAL, "polybin_set_observer: position must be finite");
    for (int a = 0; a < 3; ++a) ctx->observer[a] = pos[a];
    UwState* u = static_cast<UwState*>(ctx->ext);
    if (u) u->have_l = false;   // the local Fisher matrix belongs to the previous observer
    return POLYBIN_OK;
}

// Unwindowed P_ell with a local line of sight: p_num of eq. pk-num-fft, p = F^-1 p_num with the local Fisher,
// physical units p V / N.
template <typename T>
static int pk_unwindowed_local_t(polybin_ctx* ctx, const float* d, const float* w, double* pk_out, double* pnum_out) {
    int rc;
    if ((rc = uw_alloc<T>(ctx, false))) return rc;
    if ((rc = uw_alloc_local<T>(ctx, false))) return rc;
    UwState* u = static_cast<UwState*>(ctx->ext);
    const int na = ctx->nell * ctx->nb;
    std::vector<double> pnum;
    if ((rc = pk_numerator_local_t<T>(ctx, d, w, pnum))) return rc;
    if (pnum_out) std::memcpy(pnum_out, pnum.data(), sizeof(double) * na);
    if (!pk_out) return POLYBIN_OK;
    if (!u->have_l)
        return fail(ctx, POLYBIN_ENOTREADY, "polybin_pk_unwindowed_local: run polybin_fisher(POLYBIN_FISHER_PK_LOCAL) first");
    std::vector<double> x;
    if ((rc = apply_inverse(ctx, u->dFl_inv, na, pnum, x))) return rc;
    for (int i = 0; i < na; ++i) pk_out[i] = x[i] * ctx->vol / (double)ctx->ncell;
    return POLYBIN_OK;
}

extern "C" int polybin_pk_unwindowed_local(polybin_ctx* ctx, const float* d_dev, const float* w_dev, double* pk_out,
                                           double* pnum_out) {
    int rc = check_uw_args(ctx, d_dev, w_dev, "polybin_pk_unwindowed_local");
    if (rc) return rc;
    return ctx->prec == POLYBIN_FP64 ? pk_unwindowed_local_t<double>(ctx, d_dev, w_dev, pk_out, pnum_out)
                                     : pk_unwindowed_local_t<float>(ctx, d_dev, w_dev, pk_out, pnum_out);
}

extern "C" int polybin_pk_bias(polybin_ctx* ctx, const float* n2_dev, const float* w_dev, int which, int n_mc,
                               unsigned long long seed, double* bias_out) {
    if (!ctx || (which != 0 && which != 3) || n_mc < 0) return fail(ctx, POLYBIN_EINVAL, "polybin_pk_bias: which in {0, 3}, n_mc >= 0");
    int rc;
    if ((rc = ctx->prec == POLYBIN_FP64 ? uw_alloc<double>(ctx, false) : uw_alloc<float>(ctx, false))) return rc;
    UwState* u = static_cast<UwState*>(ctx->ext);
    if (n_mc == 0) {
        u->pbias[which].clear();
        return POLYBIN_OK;
    }
    if ((rc = check_uw_args(ctx, n2_dev, which == 0 ? w_dev : n2_dev, "polybin_pk_bias"))) return rc;
    if (which == 3 && !opt_hash(ctx))
        return fail(ctx, POLYBIN_ENOTREADY, "polybin_pk_bias(POLYBIN_FISHER_PK_OPT): call polybin_set_optimal first");
    std::vector<double> b;
    if ((rc = ctx->prec == POLYBIN_FP64 ? pk_bias_t<double>(ctx, n2_dev, w_dev, which, n_mc, seed, b)
                                        : pk_bias_t<float>(ctx, n2_dev, w_dev, which, n_mc, seed, b)))
        return rc;
    u->pbias[which] = b;
    if (bias_out) std::memcpy(bias_out, b.data(), sizeof(double) * b.size());
    return POLYBIN_OK;
}

extern "C" int polybin_pk_unwindowed_opt(polybin_ctx* ctx, const float* d_dev, double* pk_out, double* pnum_out) {
    int rc = check_uw_args(ctx, d_dev, d_dev, "polybin_pk_unwindowed_opt");
    if (rc) return rc;
    return ctx->prec == POLYBIN_FP64 ? pk_unwindowed_opt_t<double>(ctx, d_dev, pk_out, pnum_out)
                                     : pk_unwindowed_opt_t<float>(ctx, d_dev, pk_out, pnum_out);
}

extern "C" int polybin_pk_unwindowed(polybin_ctx* ctx, const float* d_dev, const float* w_dev, double* pk_out, double* pnum_out) {
    int rc = check_uw_args(ctx, d_dev, w_dev, "polybin_pk_unwindowed");
    if (rc) return rc;
    return ctx->prec == POLYBIN_FP64 ? pk_unwindowed_t<double>(ctx, d_dev, w_dev, pk_out, pnum_out)
                                     : pk_unwindowed_t<float>(ctx, d_dev, w_dev, pk_out, pnum_out);
}

extern "C" int polybin_bk_unwindowed(polybin_ctx* ctx, const float* d_dev, const float* w_dev, const float* mocks_dev,
                                     int n_mocks, double* bk_out, double* bnum_out, double* lin_out) {
    int rc = check_uw_args(ctx, d_dev, w_dev, "polybin_bk_unwindowed");
    if (rc) return rc;
    if (n_mocks < 0 || (n_mocks > 0 && (!mocks_dev || !is_device_ptr(mocks_dev))))
        return fail(ctx, POLYBIN_EINVAL, "polybin_bk_unwindowed: mocks must be device memory when n_mocks > 0");
    return ctx->prec == POLYBIN_FP64 ? bk_unwindowed_t<double>(ctx, d_dev, w_dev, mocks_dev, n_mocks, bk_out, bnum_out, lin_out)
                                     : bk_unwindowed_t<float>(ctx, d_dev, w_dev, mocks_dev, n_mocks, bk_out, bnum_out, lin_out);
}

extern "C" int polybin_bk_bias(polybin_ctx* ctx, const float* n3_dev, const float* d2_dev, const float* d_dev,
                               const float* w_dev, int n_mc, unsigned long long seed, double* bias_out) {
    int rc = check_uw_args(ctx, n3_dev, d2_dev, "polybin_bk_bias");
    if (rc || (rc = check_uw_args(ctx, d_dev, w_dev, "polybin_bk_bias"))) return rc;
    if (n_mc < 1 || !bias_out) return fail(ctx, POLYBIN_EINVAL, "polybin_bk_bias: n_mc >= 1 and bias_out required");
    std::vector<double> b;
    if ((rc = ctx->prec == POLYBIN_FP64 ? bk_bias_t<double>(ctx, n3_dev, d2_dev, d_dev, w_dev, n_mc, seed, b)
                                        : bk_bias_t<float>(ctx, n3_dev, d2_dev, d_dev, w_dev, n_mc, seed, b)))
        return rc;
    std::memcpy(bias_out, b.data(), sizeof(double) * b.size());
    return POLYBIN_OK;
}

extern "C" int polybin_bk_unwindowed_shot(polybin_ctx* ctx, const float* d_dev, const float* w_dev, const float* mocks_dev,
                                          int n_mocks, const float* n3_dev, const float* d2_dev, int n_mc,
                                          unsigned long long seed, double* bk_out, double* bnum_out, double* bias_out) {
    int rc = check_uw_args(ctx, d_dev, w_dev, "polybin_bk_unwindowed_shot");
    if (rc || (rc = check_uw_args(ctx, n3_dev, d2_dev, "polybin_bk_unwindowed_shot"))) return rc;
    if (n_mocks < 0 || (n_mocks > 0 && (!mocks_dev || !is_device_ptr(mocks_dev))) || n_mc < 1)
        return fail(ctx, POLYBIN_EINVAL, "polybin_bk_unwindowed_shot: bad mocks or n_mc < 1");
    if ((rc = ensure_triplets(ctx))) return rc;
    std::vector<double> b;
    if ((rc = ctx->prec == POLYBIN_FP64 ? bk_bias_t<double>(ctx, n3_dev, d2_dev, d_dev, w_dev, n_mc, seed, b)
                                        : bk_bias_t<float>(ctx, n3_dev, d2_dev, d_dev, w_dev, n_mc, seed, b)))
        return rc;
    if (bias_out) std::memcpy(bias_out, b.data(), sizeof(double) * b.size());
    return ctx->prec == POLYBIN_FP64
               ? bk_unwindowed_t<double>(ctx, d_dev, w_dev, mocks_dev, n_mocks, bk_out, bnum_out, nullptr, b.data())
               : bk_unwindowed_t<float>(ctx, d_dev, w_dev, mocks_dev, n_mocks, bk_out, bnum_out, nullptr, b.data());
}

extern "C" int polybin_bk_ideal_multipoles_local(polybin_ctx* ctx, const float* delta, int batch, int lmax_b,
                                                 double* bk_out) {
    if (!ctx || !delta || !bk_out || batch < 0 || lmax_b < 0 || lmax_b > 4 || lmax_b % 2)
        return fail(ctx, POLYBIN_EINVAL, "polybin_bk_ideal_multipoles_local: bad argument (lmax_b in {0, 2, 4})");
    return ctx->prec == POLYBIN_FP64 ? bk_multipoles_local_t<double>(ctx, delta, batch, lmax_b, bk_out)
                                     : bk_multipoles_local_t<float>(ctx, delta, batch, lmax_b, bk_out);
}

extern "C" int polybin_solve(polybin_ctx* ctx, const double* A, int n, const double* B, int nrhs, double* X) {
    if (!ctx || !A || !B || !X || n < 1 || nrhs < 1) return fail(ctx, POLYBIN_EINVAL, "polybin_solve: bad argument");
    return gpu_solve(ctx, A, n, B, nrhs, X);
}
