/*
 * bf_filter.h -- C ABI of the fast-convolution filter of libbf (GB300, sm_103a).
 *
 * The operation (Sec. III, the filter equation and Fig. 4): for each block s
 * of N = 2048 complex samples,
 *     y = IFFT( MULT( FFT(s) ) ),
 * where MULT is the pointwise product with the FFT of the filter sequence h
 * and all transforms have size 2048. Readings: FFT is the unnormalised DFT
 * X[k] = sum_n x[n] e^{-2 pi i n k / N}; IFFT carries the 1/N. The result is
 * then the circular convolution y[n] = sum_m h[m] s[(n - m) mod N].
 *
 * Conventions as in bf.h: complex values are interleaved FP32 pairs
 * ("complex64"); "_dev" pointers are device memory owned by the caller;
 * every call returns a bf_status, never aborts, and is asynchronous on
 * `stream` (a cudaStream_t, NULL = legacy default stream) unless stated.
 * A filter object is not thread-safe (one host thread at a time).
 *
 * Arithmetic: FP32 throughout (FP32 twiddles rounded from FP64 values, FP32
 * butterflies), one fused kernel per call: each block is read once, both
 * transforms and the product run on chip, and y is written once.
 */
#ifndef BF_FILTER_H
#define BF_FILTER_H

#include <stdint.h>

#include "bf.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bf_filter_s *bf_filter;

/* Create a filter on the current CUDA device for transforms of n points.
 * n must be 2048 (Sec. III); BF_EINVAL otherwise (checked before any CUDA
 * call), BF_ECUDA without a usable device. The filter owns its twiddle table
 * and the filter spectrum. No filter sequence is set yet. */
bf_status bf_filter_create(int n, bf_filter *out);

/* Free the filter (synchronises the device first). NULL is accepted. */
bf_status bf_filter_destroy(bf_filter filter);

/* Text of the filter's last error ("" if none); NULL gives the last error of
 * a failed bf_filter_create. */
const char *bf_filter_last_error(bf_filter filter);

/* Set the filter sequence: h_dev holds n_taps complex64 taps (8-byte
 * aligned), 1 <= n_taps <= n, zero-padded to n. The spectrum H = FFT(h) is
 * computed on the device with the library's own forward transform, ordered on
 * `stream`; later calls on other streams must be ordered after it. h_dev may
 * be freed once `stream` has passed this call. */
bf_status bf_filter_set_taps(bf_filter filter, const void *h_dev, int n_taps, void *stream);

/* Copy the current spectrum H = FFT(h), n complex64 values, to H_dev (8-byte
 * aligned). BF_ENOTFOUND if no filter sequence was set. */
bf_status bf_filter_spectrum(bf_filter filter, void *H_dev, void *stream);

/* y = IFFT(H * FFT(s)) for n_sig blocks: s_dev and y_dev hold n_sig x n
 * complex64 values, block-major (block q at q*n*8 bytes), 16-byte aligned.
 * y_dev may equal s_dev (each block is read completely before it is
 * written); other overlaps are not allowed. n_sig = 0 is a no-op.
 * BF_ENOTFOUND if no filter sequence was set. */
bf_status bf_filter_apply(bf_filter filter, const void *s_dev, int64_t n_sig, void *y_dev, void *stream);

/* The same with s and y in HOST memory (best pinned): blocks are copied in,
 * filtered and copied out in chunks over internal copy-in, compute and
 * copy-out streams. Ordered after `stream`; `stream` is ordered after its
 * completion (synchronise `stream` before reading y_host). Consecutive calls
 * on different streams (with different host buffers) pipeline: the internal
 * staging ring orders every reuse across calls. */
bf_status bf_filter_apply_host(bf_filter filter, const void *s_host, int64_t n_sig, void *y_host,
                               void *stream);

/* Declare (independent = 1) that none of the launches of this library
 * (bf_filter_apply*, bf_apply_batch*, bf_batch_launch*) enqueued on the stream
 * since its last other operation (a copy, another kernel, an event wait)
 * writes the s of the following bf_filter_apply calls -- as when the signals
 * are filled by copies, not filtered in place by those launches. A
 * call then reads and transforms s while the previous launch finishes; its
 * stores of y still wait for it. A wrong declaration gives wrong results.
 * Default 0 (s is read after the previous launch completes). The host-buffer
 * path always orders its own copies. BF_EINVAL unless independent is 0 or 1. */
bf_status bf_filter_set_s_independent(bf_filter filter, int32_t independent);

/* ------------------------------------------------------------------ building blocks
 * The paper's optimizer picks, per size and target, the best building block
 * for an operation (Sec. IV). The filter has these blocks (variants):
 *   0 : two passes per transform (2048 = 64 x 32), one warp per block of
 *       samples, 11 warps per CTA, the spectrum read through L1
 *   1 : the same with 10 warps per CTA
 *   2, 3 : the same kernel with 8 or 6 warps per CTA and the spectrum in
 *       shared memory (up to 255 registers a thread)
 *   4 : three passes per transform (2048 = 16 x 16 x 8), 128 threads per
 *       block, 4 blocks per CTA, the next block prefetched into shared memory
 *   5 : the two-pass kernel with 12 warps per CTA, the spectrum read through
 *       L1 instead of shared memory; the default (the fastest from a few
 *       hundred blocks up on GB300)
 *   6 : two passes per transform (2048 = 32 x 64), two warps per block,
 *       32 values a lane, 8 blocks per CTA; the radix-64 pass is split over
 *       lane pairs that exchange half their values by shuffles. A block
 *       finishes in about half the time of the one-warp kernels
 * Variants 0 to 3 and 5 give bit-identical results; variants 4 and 6 round
 * differently (other factorisations) within the same FP32 accuracy. The
 * spectrum of the taps is always computed the same way, whatever the
 * variant. */

/* Select the variant used by bf_filter_apply and bf_filter_apply_host
 * (BF_EINVAL outside [0, 7)). */
bf_status bf_filter_set_variant(bf_filter filter, int32_t variant);

/* The variant in use (-1 for a NULL filter). */
int32_t bf_filter_get_variant(bf_filter filter);

/* Time every variant on this GPU on n_sig synthetic blocks (1 <= n_sig <=
 * 2^20; scratch of 2 x n_sig x 16 KB is allocated and freed here; the best
 * of 3 rounds of 10 back-to-back launches, made as bf_filter_apply would
 * make them: with s independent if bf_filter_set_s_independent declared it,
 * which lets each launch's prologue overlap the previous launch and favours
 * other variants on small batches) and select the fastest. Every
 * variant computes in FP32 to the same accuracy, but variants 4 and 6 round
 * differently from the others, so tuning can change low-order result bits.
 * Runs on `stream` and synchronises it. BF_ENOTFOUND if no taps are set. */
bf_status bf_filter_autotune(bf_filter filter, int64_t n_sig, void *stream);

/* The tuned time of a variant in microseconds per launch (0 if not timed)
 * and the n_sig it was timed on. Either pointer may be NULL. */
bf_status bf_filter_tune_query(bf_filter filter, int32_t variant, double *us_per_launch, int64_t *n_sig);

/* Save / load the filter's choice and timings as JSON ("libbf-tune-2",
 * "kind": "filter") with the target it was measured on (device name,
 * compute capability, SM count). bf_filter_tune_load refuses (BF_EINVAL,
 * the filter unchanged) a table from another target or of another kind. */
bf_status bf_filter_tune_save(bf_filter filter, const char *path);
bf_status bf_filter_tune_load(bf_filter filter, const char *path);

/* Number of kernel launches issued by this filter so far. */
int64_t bf_filter_launch_count(bf_filter filter);

#ifdef __cplusplus
}
#endif

#endif /* BF_FILTER_H */
