/*
 * FP64 CPU oracle for batched complex beamforming -- TEST INFRASTRUCTURE ONLY.
 *
 * Only the tests, the smoke check and the bench's CPU-baseline leg may load
 * this library. The GPU library shares no code, header or constant with it.
 *
 * What it computes (Sec. III, beamforming equation): for every symbol block S
 * (f x b) multiplied by a precoder W (n_ant x f), the product R = W x S,
 * written row by row as the paper does: row i of R is row i of W (one antenna)
 * times S,
 *
 *     R[i][j] = sum_{k=0}^{f-1} W[i][k] * S[k][j],   0 <= i < n_ant, 0 <= j < b.
 *
 * For f = 0 the sum is empty and R = 0 (the paper lets f range from 0 to 36).
 *
 * The complex multiply-add is written out in real FP64 arithmetic,
 *     re += wr*sr - wi*si,   im += wr*si + wi*sr,
 * with k ascending and the accumulators starting at 0. Build with
 * -ffp-contract=off so that no fused multiply-add changes the rounding.
 *
 * Layouts: complex values are interleaved (re, im) doubles; W is row-major
 * n_ant x f, each S block row-major f x b, each R block row-major n_ant x b;
 * the n_blocks blocks of S and of R are contiguous.
 *
 * BFO_MUTANT (never set in a normal build) plants one deliberate mistake so
 * that the tests can show that their pins catch it.
 */
#include <stddef.h>

#ifndef BFO_MUTANT
#define BFO_MUTANT 0
#endif

int bfo_mutant_id(void) { return BFO_MUTANT; }

static void bfo_block(int n_ant, int f, int b, const double *W, const double *S, double *R)
{
    for (int i = 0; i < n_ant; i++) {
#if BFO_MUTANT == 6
        double re = 0.0, im = 0.0; /* mistake: accumulators not reset per column */
#endif
        for (int j = 0; j < b; j++) {
#if BFO_MUTANT != 6
            double re = 0.0, im = 0.0;
#endif
#if BFO_MUTANT == 2
            int kend = f > 0 ? f - 1 : 0; /* mistake: last flow dropped */
#else
            int kend = f;
#endif
            for (int k = 0; k < kend; k++) {
#if BFO_MUTANT == 5
                size_t wk = (size_t)k * n_ant + i; /* mistake: W read column-major */
                if (wk >= (size_t)n_ant * f) wk = 0;
#else
                size_t wk = (size_t)i * f + k;
#endif
#if BFO_MUTANT == 3
                size_t sk = (size_t)j * f + k; /* mistake: S read transposed */
#else
                size_t sk = (size_t)k * b + j;
#endif
                double wr = W[2 * wk], wi = W[2 * wk + 1];
                double sr = S[2 * sk], si = S[2 * sk + 1];
#if BFO_MUTANT == 1
                re += wr * sr + wi * si; /* mistake: sign of the cross term */
                im += wr * si + wi * sr;
#elif BFO_MUTANT == 4
                re += wr * sr + wi * si; /* mistake: W conjugated */
                im += wr * si - wi * sr;
#else
                re += wr * sr - wi * si;
                im += wr * si + wi * sr;
#endif
            }
            size_t rk = (size_t)i * b + j;
#if BFO_MUTANT == 7
            R[2 * rk] = im; /* mistake: real and imaginary parts swapped */
            R[2 * rk + 1] = re;
#else
            R[2 * rk] = re;
            R[2 * rk + 1] = im;
#endif
        }
    }
}

/* R_n = W x S_n for n_blocks consecutive blocks sharing one precoder W. */
void bfo_apply_blocks(int n_ant, int f, int b, long long n_blocks,
                      const double *W, const double *S, double *R)
{
    const size_t s_stride = (size_t)2 * f * b;
    const size_t r_stride = (size_t)2 * n_ant * b;
#pragma omp parallel for schedule(static)
    for (long long n = 0; n < n_blocks; n++)
        bfo_block(n_ant, f, b, W, S + (size_t)n * s_stride, R + (size_t)n * r_stride);
}

/* Use n OpenMP threads from now on (no effect without OpenMP). */
void bfo_set_num_threads(int n)
{
#ifdef _OPENMP
    extern void omp_set_num_threads(int);
    if (n > 0)
        omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* Number of OpenMP threads the oracle uses (1 when built without OpenMP). */
int bfo_num_threads(void)
{
    int n = 1;
#pragma omp parallel
    {
#pragma omp single
        {
#ifdef _OPENMP
            extern int omp_get_num_threads(void);
            n = omp_get_num_threads();
#endif
        }
    }
    return n;
}
