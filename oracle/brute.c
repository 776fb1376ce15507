/* Brute-force closed-triangle sums on a periodic grid (oracle pin; test infrastructure only).
 *
 * For every ordered pair of modes (k1, k2) with |k1| in bin a and |k2| in bin b, the third mode
 * k3 = -(k1 + k2) (mod the grid) closes the triangle; if |k3| lies in bin c the pair contributes
 * 1 to count[a][b][c] and Re(D(k1) D(k2) D(k3)) to sdd[a][b][c].  This is the direct definition of
 * the closed-triangle integral int_{k123=0} Theta_a Theta_b Theta_c (...) of Sec. 4.1 (eqs. N-ell-def,
 * ideal-bk) on the discrete grid, with no FFTs.  ``brute_bk3`` takes three spectra, one per slot
 * (D1(k1) D2(k2) D3(k3)), for the mixed sums of the bispectrum linear term (Sec. 4.3.2).  Bins are half-open [e_b, e_{b+1}) in |k| = kf sqrt(|n|^2),
 * k = 0 excluded.  D is the full complex DFT in numpy fftn order (re and im arrays, C order).
 */
#include <math.h>
#include <stdlib.h>

static int bin_of(long s, double kf, const double* edges, int nb) {
    if (s <= 0) return -1;
    double k = kf * sqrt((double)s);
    if (k < edges[0]) return -1;
    for (int b = 0; b < nb; ++b)
        if (k >= edges[b] && k < edges[b + 1]) return b;
    return -1;
}

static int freq(int i, int n) { return i < n / 2 ? i : i - n; }
static int wrap(int v, int n) { v %= n; return v < 0 ? v + n : v; }

int brute_bk3(int n0, int n1, int n2, double kf, const double* edges, int nb,
              const double* r1, const double* i1_, const double* r2, const double* i2_,
              const double* r3, const double* i3_, double* count, double* sdd) {
    long ncell = (long)n0 * n1 * n2;
    int* bin = (int*)malloc(sizeof(int) * ncell);
    if (!bin) return -1;
    for (int i = 0; i < n0; ++i)
        for (int j = 0; j < n1; ++j)
            for (int k = 0; k < n2; ++k) {
                long a = freq(i, n0), b = freq(j, n1), c = freq(k, n2);
                bin[((long)i * n1 + j) * n2 + k] = bin_of(a * a + b * b + c * c, kf, edges, nb);
            }
    long nbin = 0;
    for (long m = 0; m < ncell; ++m) nbin += bin[m] >= 0;
    long* list = (long*)malloc(sizeof(long) * (nbin ? nbin : 1));
    if (!list) { free(bin); return -1; }
    long q = 0;
    for (long m = 0; m < ncell; ++m) if (bin[m] >= 0) list[q++] = m;
    long nb3 = (long)nb * nb * nb;
    for (long t = 0; t < nb3; ++t) { count[t] = 0.0; if (sdd) sdd[t] = 0.0; }
    for (long p = 0; p < nbin; ++p) {
        long m1 = list[p];
        int i1 = (int)(m1 / ((long)n1 * n2)), j1 = (int)((m1 / n2) % n1), k1 = (int)(m1 % n2);
        int a = bin[m1];
        for (long r = 0; r < nbin; ++r) {
            long m2 = list[r];
            int i2 = (int)(m2 / ((long)n1 * n2)), j2 = (int)((m2 / n2) % n1), k2 = (int)(m2 % n2);
            int i3 = wrap(-(i1 + i2), n0), j3 = wrap(-(j1 + j2), n1), k3 = wrap(-(k1 + k2), n2);
            long m3 = ((long)i3 * n1 + j3) * n2 + k3;
            int c = bin[m3];
            if (c < 0) continue;
            long t = ((long)a * nb + bin[m2]) * nb + c;
            count[t] += 1.0;
            if (sdd) {
                double xr = r1[m1] * r2[m2] - i1_[m1] * i2_[m2];
                double xi = r1[m1] * i2_[m2] + i1_[m1] * r2[m2];
                sdd[t] += xr * r3[m3] - xi * i3_[m3];
            }
        }
    }
    free(list);
    free(bin);
    return 0;
}

int brute_bk(int n0, int n1, int n2, double kf, const double* edges, int nb,
             const double* dre, const double* dim, double* count, double* sdd) {
    return brute_bk3(n0, n1, n2, kf, edges, nb, dre, dim, dre, dim, dre, dim, count, sdd);
}
