/*
 * FP64 CPU oracle for the fast-convolution filter -- TEST INFRASTRUCTURE ONLY.
 *
 * Only the tests, the smoke check and the bench's CPU-baseline leg may load
 * this code (it is linked into the same oracle library as the beamforming
 * product). The GPU library shares no code, header, table or constant with it.
 *
 * What the paper computes (Sec. III, the filter equation and Fig. 4): for a
 * signal block s of N = 2048 complex samples,
 *
 *     y = IFFT( MULT( FFT(s) ) ),
 *
 * MULT being the pointwise product with the FFT of the filter sequence h.
 * Reading (the paper gives no normalisation): the forward transform is the
 * unnormalised DFT, X[k] = sum_n x[n] e^{-2 pi i n k / N}, and the inverse
 * carries the 1/N, x[n] = (1/N) sum_k X[k] e^{+2 pi i n k / N}. With that
 * reading the filter is exactly the circular convolution of h and s
 * (convolution theorem), which this oracle evaluates by its definition:
 *
 *     y[n] = sum_{m=0}^{N-1} h[m] * s[(n - m) mod N],   0 <= n < N.
 *
 * bfo_dft evaluates the DFT itself by its definition (O(N^2) sums, the angle
 * of each term reduced exactly as the integer (n k) mod N before the cosine
 * and sine), for the filter spectrum H = DFT(h).
 *
 * Layouts: complex values are interleaved (re, im) doubles; a batch of
 * signals is signal-major, each signal N contiguous samples.
 *
 * BFO_MUTANT 8..10 (never set in a normal build) plant deliberate mistakes so
 * that the tests can show that their pins catch them.
 */
#include <math.h>
#include <stddef.h>

#ifndef BFO_MUTANT
#define BFO_MUTANT 0
#endif

static void bfo_conv_one(int n, const double *h, const double *s, double *y)
{
    for (int t = 0; t < n; t++) {
        double re = 0.0, im = 0.0;
        for (int m = 0; m < n; m++) {
#if BFO_MUTANT == 8
            int idx = (t + m) % n; /* mistake: correlation instead of convolution */
#elif BFO_MUTANT == 9
            int idx = t - m; /* mistake: no circular wrap (linear convolution, truncated) */
            if (idx < 0)
                continue;
#else
            int idx = ((t - m) % n + n) % n;
#endif
            double hr = h[2 * m], hi = h[2 * m + 1];
#if BFO_MUTANT == 10
            hi = -hi; /* mistake: filter taps conjugated */
#endif
            double sr = s[2 * idx], si = s[2 * idx + 1];
            re += hr * sr - hi * si;
            im += hr * si + hi * sr;
        }
        y[2 * t] = re;
        y[2 * t + 1] = im;
    }
}

/* y_q = h (circularly convolved with) s_q for n_sig signals of n samples. */
void bfo_circular_filter(int n, long long n_sig, const double *h, const double *s, double *y)
{
#pragma omp parallel for schedule(static)
    for (long long q = 0; q < n_sig; q++)
        bfo_conv_one(n, h, s + (size_t)q * 2 * n, y + (size_t)q * 2 * n);
}

/* The DFT by its definition, for count sequences of n samples: sign -1 gives
 * X[k] = sum_j x[j] e^{-2 pi i j k / n}; sign +1 the same sum with e^{+...}
 * (no 1/n factor). */
void bfo_dft(int n, int sign, long long count, const double *x, double *X)
{
    const double two_pi = 6.283185307179586476925286766559;
#pragma omp parallel for schedule(static)
    for (long long q = 0; q < count; q++) {
        const double *xq = x + (size_t)q * 2 * n;
        double *Xq = X + (size_t)q * 2 * n;
        for (int k = 0; k < n; k++) {
            double re = 0.0, im = 0.0;
            for (int j = 0; j < n; j++) {
                long long r = ((long long)j * k) % n;
                double a = two_pi * (double)r / (double)n;
                double c = cos(a), sn = sign * sin(a);
                double xr = xq[2 * j], xi = xq[2 * j + 1];
                re += xr * c - xi * sn;
                im += xr * sn + xi * c;
            }
            Xq[2 * k] = re;
            Xq[2 * k + 1] = im;
        }
    }
}
