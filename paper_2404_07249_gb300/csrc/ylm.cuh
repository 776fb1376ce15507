// Normalised real spherical harmonics for the local (Yamamoto) line of sight, Sec. 3.3.1: the functions Ybar_lm
// with sum_m Ybar_lm(a) Ybar_lm(b) = L_l(a.b) for unit vectors a, b.  From the addition theorem of the Legendre
// polynomials, L_l(a.b) = L_l(a_z) L_l(b_z) + 2 sum_{m>0} (l-m)!/(l+m)! P_l^m(a_z) P_l^m(b_z) cos m(phi_a - phi_b)
// with P_l^m(z) = (1 - z^2)^{m/2} d^m L_l / dz^m, one such set is
//     Ybar_l0 = L_l(z),   Ybar_l,m = c_lm d^m L_l/dz^m (z) Re (x + i y)^m,   Ybar_l,-m = c_lm d^m L_l/dz^m (z) Im (x + i y)^m,
// c_lm = sqrt(2 (l-m)! / (l+m)!), m = 1 .. l.  Every quantity the estimators use is a sum over m of products of two
// Ybar_lm of the same (l, m), so any orthonormal set with this normalisation gives the same results.
#pragma once
#include <cuda_runtime.h>

namespace pb {

// Ybar_lm(x, y, z) for a unit vector, l in {0, 2, 4}, |m| <= l (0 otherwise).
template <typename T>
__host__ __device__ inline T ybar(int ell, int m, T x, T y, T z) {
    const int am = m < 0 ? -m : m;
    if (ell == 0) return am == 0 ? T(1) : T(0);
    // (x + i y)^|m|
    T re = T(1), im = T(0);
    for (int q = 0; q < am; ++q) {
        const T r2 = re * x - im * y;
        im = re * y + im * x;
        re = r2;
    }
    const T z2 = z * z;
    T d = T(0), c = T(0);   // d^|m| L_l / dz^|m| and c_lm
    if (ell == 2) {
        if (am == 0) { d = T(0.5) * (T(3) * z2 - T(1)); c = T(1); }
        else if (am == 1) { d = T(3) * z; c = T(0.5773502691896257); }
        else if (am == 2) { d = T(3); c = T(0.28867513459481287); }
    } else if (ell == 4) {
        if (am == 0) { d = (T(35) * z2 * z2 - T(30) * z2 + T(3)) / T(8); c = T(1); }
        else if (am == 1) { d = T(0.5) * (T(35) * z2 - T(15)) * z; c = T(0.31622776601683794); }
        else if (am == 2) { d = T(0.5) * (T(105) * z2 - T(15)); c = T(0.07453559924999299); }
        else if (am == 3) { d = T(105) * z; c = T(0.019920476822239894); }
        else if (am == 4) { d = T(105); c = T(0.0070429521227376385); }
    }
    if (am == 0) return d;
    return c * d * (m > 0 ? re : im);
}

// Unit vector from the observer to the centre of cell (i, j, k), in the working precision T: centres at
// (i + 1/2) h_a - L/2 (a box centred on the origin, h_a = L / N_a); the z axis where the centre coincides with the
// observer.
template <typename T>
__host__ __device__ inline void cell_direction(long i, long j, long k, const T* h, T half_l, const T* obs, T& x, T& y,
                                               T& z) {
    const T px = (T(i) + T(0.5)) * h[0] - half_l - obs[0];
    const T py = (T(j) + T(0.5)) * h[1] - half_l - obs[1];
    const T pz = (T(k) + T(0.5)) * h[2] - half_l - obs[2];
    const T r2 = px * px + py * py + pz * pz;
    if (r2 > T(0)) {
        const T inv = T(1) / sqrt(r2);
        x = px * inv; y = py * inv; z = pz * inv;
    } else {
        x = T(0); y = T(0); z = T(1);
    }
}

}  // namespace pb
