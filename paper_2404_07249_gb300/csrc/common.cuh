// Shared device/host helpers for libpolybin (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace pb {

template <typename T> struct cplx_t;
template <> struct cplx_t<float> { using type = float2; };
template <> struct cplx_t<double> { using type = double2; };
template <typename T> using C = typename cplx_t<T>::type;

template <typename T> __host__ __device__ __forceinline__ C<T> mk(T x, T y) { C<T> r; r.x = x; r.y = y; return r; }
template <typename T> __device__ __forceinline__ C<T> add(C<T> a, C<T> b) { return mk<T>(a.x + b.x, a.y + b.y); }
template <typename T> __device__ __forceinline__ C<T> sub(C<T> a, C<T> b) { return mk<T>(a.x - b.x, a.y - b.y); }
template <typename T> __device__ __forceinline__ C<T> scl(C<T> a, T s) { return mk<T>(a.x * s, a.y * s); }
// FP32 complex sums as one packed f32x2 instruction (two round-to-nearest adds, the same values as two scalar
// adds): the butterflies of the FFT passes are mostly such sums, and the passes are bound by instruction issue.
__device__ __forceinline__ uint64_t f32x2_bits(float2 a) { return *reinterpret_cast<const uint64_t*>(&a); }
__device__ __forceinline__ float2 f32x2_val(uint64_t r) { return *reinterpret_cast<const float2*>(&r); }
template <> __device__ __forceinline__ float2 add<float>(float2 a, float2 b) {
    uint64_t r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f32x2_bits(a)), "l"(f32x2_bits(b)));
    return f32x2_val(r);
}
template <> __device__ __forceinline__ float2 sub<float>(float2 a, float2 b) {
    uint64_t r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f32x2_bits(a)), "l"(f32x2_bits(b)));
    return f32x2_val(r);
}
template <typename T> __device__ __forceinline__ C<T> mul(C<T> a, C<T> b) {
    return mk<T>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
template <typename T> __device__ __forceinline__ C<T> mulc(C<T> a, C<T> b) {
    return mk<T>(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
// multiply by i*s (s = +1 or -1): i*(x+iy) = -y + ix
template <typename T> __device__ __forceinline__ C<T> muli(C<T> a, int s) {
    return s > 0 ? mk<T>(-a.y, a.x) : mk<T>(a.y, -a.x);
}

// Integer wave number of FFT position i on an axis of length n (numpy fftfreq ordering).
__host__ __device__ __forceinline__ int freq_of(int i, int n) { return i < n / 2 ? i : i - n; }
// FFT position of wave number f on an axis of length n.
__host__ __device__ __forceinline__ int pos_of(int f, int n) { return f >= 0 ? f : f + n; }

// A contiguous range of wave numbers kept on one axis: f in [lo, lo + cnt).
struct AxisRange {
    int lo, cnt;
};

}  // namespace pb

#define PB_CUDA_OK(expr)                                                                          \
    do {                                                                                          \
        cudaError_t _e = (expr);                                                                  \
        if (_e != cudaSuccess) return pb::fail_cuda(ctx, _e, #expr, __FILE__, __LINE__);          \
    } while (0)
