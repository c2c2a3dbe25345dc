/*
 * bf.h -- C ABI of libbf, batched complex beamforming R = W x S on GB300 (sm_103a).
 *
 * The operation (Sec. III, beamforming equation and the sentences around it):
 * a precoding matrix W with one row per antenna (n_ant = 64, Sec. II) and f
 * columns, one per parallel flow (0 <= f <= 36), is applied to many symbol
 * blocks S of f rows by b = 60 resource elements; W stays constant while S
 * changes. Each block gives R = W x S (n_ant x b), i.e. for every antenna i
 *     R[i][j] = sum_{k<f} W[i][k] * S[k][j],   j < b.
 * f = 0 gives R = 0.
 *
 * Conventions shared by every entry point
 *  - Complex numbers are interleaved (re, im) FP32 pairs ("complex64").
 *  - W is row-major n_ant x f (antenna-major); an S block is row-major f x b
 *    (flow-major, b = 60 contiguous complex per flow); an R block is row-major
 *    n_ant x b. A block of S is 480*f bytes, a block of R 30,720 bytes.
 *  - Blocks that share a precoder form a group and are contiguous in S and R.
 *  - "_dev" pointers are CUDA device pointers (e.g. from PyTorch), "_host"
 *    pointers are host memory. The caller owns every buffer it passes; the
 *    library never frees or keeps them past the call except where stated.
 *  - Device buffers and byte offsets must be 16-byte aligned (BF_EINVAL).
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream). Calls that
 *    take a stream are asynchronous on it unless stated otherwise.
 *  - Every call returns a bf_status and never aborts or exits. The text of the
 *    last error of a plan is in bf_last_error(plan).
 *  - A plan is not thread-safe: one host thread at a time per plan (the
 *    serving engine serialises its own use internally).
 */
#ifndef BF_H
#define BF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    BF_OK = 0,
    BF_EINVAL = 1,     /* an argument is out of range, NULL or misaligned      */
    BF_ENOMEM = 2,     /* device or host allocation failed                      */
    BF_EBUDGET = 3,    /* a serving job is larger than the whole HBM budget     */
    BF_ECUDA = 4,      /* a CUDA runtime call failed (text in bf_last_error)   */
    BF_ETIMEOUT = 5,   /* a bounded device or host wait gave up                */
    BF_EAGAIN = 6,     /* the serving queue is full; try again                  */
    BF_EBUSY = 7,      /* the object still has work in flight                   */
    BF_ENOTREADY = 8,  /* the result is not available yet                       */
    BF_ENOTFOUND = 9   /* unknown ticket / unset precoder slot                  */
} bf_status;

/* Arithmetic of the product. All forms accumulate in FP32 and write complex64 R
 * (or the type a bf_rlayout names).
 *  BF_FP32   : plain form, FP32 fused multiply-add on the CUDA cores; S complex64.
 *  BF_FP32_3M: FP32 on the CUDA cores with three real products per complex
 *              multiply-add instead of four: per output element
 *              P1 = sum Re W Re S, P2 = sum Im W Im S,
 *              P3 = sum (Re W + Im W)(Re S + Im S),
 *              Re R = P1 - P2, Im R = (P3 - P1) - P2; S complex64.
 *  BF_BF16   : single-pass tensor-core form, operands rounded to bfloat16.
 *  BF_FP16   : single-pass tensor-core form, operands rounded to binary16.
 *  BF_BF16X3 : split form, x = hi + lo (hi = bf16(x), lo = bf16(x - hi)),
 *              R = Wh*Sh + Wh*Sl + Wl*Sh on the tensor cores.
 *  BF_TF32X3 : the same split with TF32 terms (hi = tf32(x), lo = tf32(x - hi),
 *              both rounded to nearest even; 10 fraction bits each): about
 *              2^-21 relative error per product where BF_BF16X3 has 2^-16.
 *              S complex64 only (no held form).
 * The 16-bit tensor-core forms take S either as complex64 (converted on chip,
 * no per-block scale) or "held": pre-encoded by bf_quantize_symbols with one
 * power-of-two scale per block. W is always taken from the plan's images. */
typedef enum {
    BF_FP32 = 0,
    BF_BF16 = 1,
    BF_FP16 = 2,
    BF_BF16X3 = 3,
    BF_FP32_3M = 4,
    BF_TF32X3 = 5
} bf_precision;

/* One group: n_blocks consecutive blocks that all multiply precoder prec_id.
 * s_off / r_off are BYTE offsets of the group's first block in the S and R
 * buffers (multiples of 16). For complex64 S, block n of the group starts at
 * s_off + n*480*f; for held S at s_off + n*bf_held_block_bytes(f, prec).
 * R block n starts at r_off + n*30720. */
typedef struct {
    int32_t prec_id;
    int32_t n_blocks;
    int64_t s_off;
    int64_t r_off;
} bf_group;

typedef struct bf_plan_s *bf_plan;

/* ------------------------------------------------------------------ plan */

/* Create a plan on the current CUDA device. The kernels are built for the
 * paper's shapes: n_ant must be 64, b must be 60 and 0 <= f_max <= 36
 * (Sec. III). Returns BF_EINVAL for other shapes (checked before any CUDA
 * call), BF_ECUDA if there is no usable sm_103 device. *out receives the plan.
 * The plan owns the precoder images, its work-list buffers, captured graphs,
 * the autotune table and its device status word. */
bf_status bf_plan_create(int n_ant, int f_max, int b, bf_plan *out);

/* Free the plan and everything it owns. Synchronises the device first.
 * NULL is accepted (BF_OK). BF_EBUSY (nothing freed) while a serving engine
 * created on the plan (bf_serve_create) has not been destroyed. */
bf_status bf_plan_destroy(bf_plan plan);

/* Human-readable text of the plan's last error ("" if none), copied for the
 * calling thread: valid in that thread until its next bf_last_error call,
 * also while other threads (a serving engine) use the plan. A NULL plan gives
 * this thread's last plan-less error (creation). */
const char *bf_last_error(bf_plan plan);

/* Static name of a status code. */
const char *bf_status_string(bf_status s);

/* Reads and clears the plan's device status word, which kernels set when a
 * bounded on-chip wait gives up (they then stop early, leaving R incomplete).
 * Synchronises the device. BF_OK or BF_ETIMEOUT. */
bf_status bf_device_status(bf_plan plan);

/* Self-test of the failure detection in the kernels' pipelines. Launches one
 * CTA in which two roles wait, through the same bounded mbarrier wait the
 * product kernels use, on barriers that nothing completes: the first gives up
 * after the wait limit (2 s), raises the CTA's abort flag and sets the plan's
 * device status word; the second, which starts waiting 1 s later, leaves
 * through the abort flag before its own limit. Nothing faults or hangs and the
 * context stays usable. Synchronises, then writes to out_host[4]: first role
 * gave up (1/0), its wait in ms, second role left early (1/0), its wait in
 * ms. The status word stays set for the next bf_device_status (BF_ETIMEOUT). */
bf_status bf_selftest_wait_timeout(bf_plan plan, int32_t *out_host);

/* ------------------------------------------------------------------ precoders */

/* Set precoder slots first_id .. first_id+n_prec-1 (Sec. III: W is constant
 * across many S, so it is converted once here and reused).
 *  W_dev  : n_prec precoders packed back to back, precoder p row-major
 *           n_ant x f_host[p] complex64 (device, 8-byte aligned).
 *  f_host : f of each precoder, 0 <= f <= f_max.
 * Builds, on `stream`, every device image the kernels read: planar FP32,
 * bfloat16 hi/lo and binary16 in the tensor cores' shared-memory layout, with
 * a power-of-two scale per precoder (2^ceil(log2 max(|Re|,|Im|))). Slots grow
 * on demand; growing synchronises the device. Later launches that read these
 * slots must be ordered after `stream`. W_dev may be freed once `stream` has
 * passed this call. */
bf_status bf_set_precoders(bf_plan plan, const void *W_dev, const int32_t *f_host,
                           int32_t n_prec, int32_t first_id, void *stream);

/* The images bf_set_precoders made of one precoder slot, copied to host
 * memory (inspection and tests; synchronises the device):
 *  BF_IMG_FP32   : FP32 planes for the CUDA-core kernels, float index k*64 + i
 *                  of plane 0 = Re W[i][k], plane 1 = Im W[i][k], plane 2 =
 *                  Re + Im (FP32 sum); 3 * 64 * f floats.
 *  BF_IMG_BF16X2 : bf16 hi image then lo image of the real-block operand B
 *                  (row n = 2i + c, column kk = 2k + c': row 2i = (Re, -Im),
 *                  row 2i + 1 = (Im, Re), all divided by the slot's scale),
 *                  K = 2f rounded up to 16, each in the layout of held S
 *                  (bf_held_block_bytes) with 128 rows; 2 * 128 * K * 2 bytes.
 *  BF_IMG_FP16   : the same operand in fp16; 128 * K * 2 bytes.
 *  BF_IMG_TF32X2 : tf32 hi then lo image of the operand, K = 2f rounded up to
 *                  8, 32-bit values at (row/8)*32*K + (col/4)*128 + (row%8)*16
 *                  + (col%4)*4; 2 * 128 * K * 4 bytes.
 *  BF_IMG_SCALE  : the slot's power-of-two scale, one float.
 * With host_out NULL only *bytes_out is set. BF_ENOTFOUND for an unset slot,
 * BF_EINVAL for an unknown kind or capacity < the image size. */
typedef enum { BF_IMG_FP32 = 0, BF_IMG_BF16X2 = 1, BF_IMG_FP16 = 2, BF_IMG_TF32X2 = 3, BF_IMG_SCALE = 4 } bf_image;
bf_status bf_get_precoder_image(bf_plan plan, int32_t slot, bf_image kind, void *host_out, int64_t capacity,
                                int64_t *bytes_out);

/* Grow the precoder store to at least n_slots slots now, so that later
 * bf_set_precoders calls on slots below n_slots never reallocate it (growing
 * synchronises the device and copies every image, which a latency-bound
 * caller such as a serving loop should do before it starts). BF_EINVAL for
 * n_slots < 0 or above 2^24; BF_ENOMEM if the store cannot grow. */
bf_status bf_reserve_precoders(bf_plan plan, int32_t n_slots);

/* Size every buffer of the plan's work-list ring for batches of up to
 * max_blocks blocks now. A call whose work list outgrows a ring buffer
 * otherwise allocates a bigger one on the spot (pinned host and device
 * memory; the old one is kept until the plan is destroyed, so nothing
 * synchronises the device); a serving loop reserves its largest merged
 * launch before it starts. BF_EINVAL for max_blocks < 0 or above 2^30. */
bf_status bf_reserve_worklists(bf_plan plan, int64_t max_blocks);

/* ------------------------------------------------------------------ held symbols */

/* Bytes of one held (pre-encoded) S block for precision prec at f flows:
 * terms * 128 * K, K = 2f rounded up to a multiple of 16, terms = 2 for
 * BF_BF16X3 and 1 for BF_BF16 / BF_FP16; 0 for the FP32 forms or f out of range.
 * Layout of a term: 64 rows (resource element j; rows 60..63 are zero) by K
 * columns (column 2k = Re S[k][j], 2k+1 = Im S[k][j], zero beyond 2f), stored
 * as 8x8 tiles of 16-bit values: element (row, col) at byte
 * (row/8)*16*K + (col/8)*128 + (row%8)*16 + (col%8)*2. For BF_BF16X3 the hi
 * term comes first, then the lo term. */
int64_t bf_held_block_bytes(int f, bf_precision prec);

/* Encode complex64 S blocks for a tensor-core precision ("held" S).
 *  S_dev      : complex64 S; group g's blocks at groups[g].s_off (bytes).
 *  q_off_host : per group, the byte offset of its first held block in Sq_dev
 *               (multiple of 16); its blocks follow at bf_held_block_bytes.
 *  scale_dev  : one float per block, in group order (block n of group g at
 *               index sum_{h<g} n_blocks[h] + n): the power of two that the
 *               encoded values are multiplied by to give S back.
 * Per block: scale = 2^ceil(log2 m), m = max over the block of |Re| and |Im|
 * (1 when m = 0); each value x/scale is rounded to nearest even in the target
 * format; BF_BF16X3 stores hi = bf16(x/scale) and lo = bf16(x/scale - hi). */
bf_status bf_quantize_symbols(bf_plan plan, const void *S_dev, const bf_group *groups,
                              int32_t n_groups, bf_precision prec, void *Sq_dev,
                              const int64_t *q_off_host, float *scale_dev, void *stream);

/* ------------------------------------------------------------------ the product */

/* R = W x S for every block of every group, in one persistent launch on
 * `stream` (Sec. III).
 *  S_dev     : complex64 S (scale_dev == NULL) or held S from
 *              bf_quantize_symbols (scale_dev != NULL; BF_BF16, BF_FP16 and
 *              BF_BF16X3 only). Group offsets as in bf_group.
 *  groups    : host array, read during the call only.
 *  R_dev     : complex64 R; every element of every listed block is written
 *              (zeros for f = 0).
 * The host builds a work list (tiles of up to two blocks of one group, each
 * CTA a cost-balanced run of tiles) and uploads it to a plan-owned buffer;
 * the launch then reads it. Calls on one plan must not overlap in host
 * threads; launches on different streams may overlap on the device only if
 * each call's work list is not still being read, which the plan guarantees by
 * keeping one work-list buffer per call in flight (a ring; the oldest is
 * reused after its launch has completed). */
bf_status bf_apply_batch(bf_plan plan, const void *S_dev, const float *scale_dev,
                         const bf_group *groups, int32_t n_groups, bf_precision prec,
                         void *R_dev, void *stream);

/* Output layout and type of R. The stage after beamforming works per antenna
 * (each antenna's OFDM modulator takes that antenna's subcarriers as one
 * vector, Sec. II-III), so R can be written straight into such a layout
 * instead of block-major complex64. Element (block n of a group, antenna i,
 * resource element j) is stored at byte
 *     r_off + n*block_stride + i*row_stride + j*esize
 * of R_dev, where r_off is the group's offset and esize is 8 for BF_R_C64
 * (interleaved FP32) and 4 for BF_R_BF16 / BF_R_FP16 (an interleaved pair of
 * 16-bit values, each rounded to nearest even from the FP32 accumulator).
 * The packed default (layout == NULL) is {480, 30720, BF_R_C64}.
 * Antenna-major, subcarrier-contiguous output of T blocks, say, uses
 *     row_stride = T*60*esize, block_stride = 60*esize,
 *     r_off of a group = (index of its first block)*60*esize,
 * so antenna i's T*60 resource elements are one contiguous row.
 * Rules (BF_EINVAL otherwise): both strides positive multiples of 16, each at
 * least 60*esize. The caller sizes R_dev and guarantees that no two listed
 * elements share an address (not checked). */
typedef enum { BF_R_C64 = 0, BF_R_BF16 = 1, BF_R_FP16 = 2 } bf_rtype;
typedef struct {
    int64_t row_stride;    /* bytes between antennas i and i+1 of one block */
    int64_t block_stride;  /* bytes between blocks n and n+1 of one group   */
    int32_t rtype;         /* bf_rtype                                      */
    int32_t reserved;      /* must be 0                                     */
} bf_rlayout;

/* bf_apply_batch with an explicit R layout (NULL = the packed default). The
 * product and its FP32 accumulation are unchanged; only the store differs. */
bf_status bf_apply_batch_rl(bf_plan plan, const void *S_dev, const float *scale_dev,
                            const bf_group *groups, int32_t n_groups, bf_precision prec,
                            void *R_dev, const bf_rlayout *layout, void *stream);

/* The same product with S and R in HOST memory (best pinned). S is copied in,
 * the product runs, R is copied out, pipelined in chunks of groups (S + R of
 * 4 MiB first, doubling up to 32 MiB by default; bf_set_host_chunks) over
 * three internal streams (copy in, compute, copy out), so both directions of
 * the host link stay busy.
 * Ordered after `stream`; `stream` is ordered after its completion
 * (synchronise `stream` before reading R_host). Group offsets refer to the
 * host buffers. Consecutive calls on different streams (with different host
 * buffers) pipeline: a call's copy-in overlaps the previous call's copy-out,
 * the internal staging ring ordering every reuse. */
bf_status bf_apply_batch_host(bf_plan plan, const void *S_host, const bf_group *groups,
                              int32_t n_groups, bf_precision prec, void *R_host,
                              void *stream);

/* Chunk sizes (S + R bytes) of bf_apply_batch_host: the first chunk, small so
 * that the copy-out starts early, and the largest, to which chunks double.
 * Defaults 4 MiB and 32 MiB. A caller that keeps several calls in flight on
 * different streams moves bytes faster with larger chunks (on GB300 the
 * full-band round trip took 0.685 ms per call with 32 MiB and 0.672 ms with
 * 8 and 64 MiB; one call at a time, 0.726 and 0.745 ms). BF_EINVAL unless
 * 64 KiB <= first_bytes <= max_bytes <= 16 GiB. */
bf_status bf_set_host_chunks(bf_plan plan, int64_t first_bytes, int64_t max_bytes);

/* A prepared batch: the work list is built and uploaded once, and the one
 * persistent launch is also captured in a CUDA graph. Arguments as
 * bf_apply_batch; the buffers must stay valid for the batch's lifetime.
 *  bf_batch_launch       : launches the kernel directly on `stream` (the
 *                          cheapest form; it may itself be captured into a
 *                          caller's graph).
 *  bf_batch_launch_graph : replays the batch's own captured graph on `stream`.
 * Both compute the same bits. */
typedef struct bf_batch_s *bf_batch;
bf_status bf_batch_create(bf_plan plan, const void *S_dev, const float *scale_dev,
                          const bf_group *groups, int32_t n_groups, bf_precision prec,
                          void *R_dev, bf_batch *out);
/* bf_batch_create with an explicit R layout (as bf_apply_batch_rl). */
bf_status bf_batch_create_rl(bf_plan plan, const void *S_dev, const float *scale_dev,
                             const bf_group *groups, int32_t n_groups, bf_precision prec,
                             void *R_dev, const bf_rlayout *layout, bf_batch *out);
bf_status bf_batch_launch(bf_batch batch, void *stream);
bf_status bf_batch_launch_graph(bf_batch batch, void *stream);
bf_status bf_batch_destroy(bf_batch batch);

/* Declare (independent = 1) that none of the launches of this library
 * (bf_apply_batch*, bf_batch_launch*, bf_filter_apply*) enqueued on the
 * stream since its last other operation (a copy, another kernel, an event
 * wait) writes this batch's S or held-S scales -- as when S lives in its own
 * buffers, filled by copies or other kernels, in a double-buffered pipeline.
 * (Those launches may release the next launch before they complete; other
 * work does not.) bf_batch_launch then
 * loads S and computes while those launches finish; only its stores of R wait
 * for them (R may overlap what they read or write). A wrong declaration gives
 * wrong results. Default 0. The captured graph (bf_batch_launch_graph) keeps
 * the default. BF_EINVAL unless independent is 0 or 1. */
bf_status bf_batch_set_s_independent(bf_batch batch, int32_t independent);

/* ------------------------------------------------------------------ scheduler */

/* One work item of a launch: up to two consecutive blocks of one group. */
typedef struct {
    int64_t s_off;       /* byte offset of the first block in S                  */
    int64_t r_off;       /* byte offset of the first block in R                  */
    int32_t prec_id;     /* precoder slot                                        */
    int32_t first_block; /* index of the first block in group order              */
    int16_t f;           /* flows of the precoder                                */
    int16_t n_blocks;    /* 1 or 2                                               */
    int32_t flags;       /* 1: first tile of its precoder in its CTA's run;
                            2: last such tile (tiles with f > 0 only)            */
} bf_tile;

/* The work-list scheduler that bf_apply_batch runs on the host, exposed as a
 * pure host function (no CUDA call). The groups (Sec. III: many S per
 * constant W) are cut into tiles of up to two blocks, in group order, and the
 * tiles are split into at most max_cta contiguous runs of about equal cost
 * (bytes of S read and R written, optionally weighted per f by the autotune
 * table; here the weights are 1), one run per CTA, so each CTA loads a
 * precoder once per run.
 *  f_of_slot : f of each precoder slot (n_slots entries).
 *  tiles_out : NULL to query the tile count; else room for max_tiles tiles.
 *  cta_begin_out : room for max_cta + 1 entries; CTA c runs tiles
 *                  [cta_begin_out[c], cta_begin_out[c+1]).
 *  *n_cta_out receives the number of CTAs.
 * Returns the number of tiles, or -BF_EINVAL. */
int32_t bf_schedule(const int32_t *f_of_slot, int32_t n_slots, const bf_group *groups, int32_t n_groups,
                    bf_precision prec, int32_t held, int32_t max_cta, bf_tile *tiles_out,
                    int32_t max_tiles, int32_t *cta_begin_out, int32_t *n_cta_out);

/* ------------------------------------------------------------------ autotuner */

/* Tune `prec` on this GPU, the way the paper's optimizer picks the best
 * building block per size and target (Sec. IV). For each f bucket ([0],
 * [1,8], [9,16], [17,24], [25,36], measured at f = 0, 8, 16, 24, 36) it times
 * synthetic complex64 batches of sm_count*8 and sm_count*32 blocks, 14 blocks
 * per precoder, with tiles of 1 and of 2 blocks. It keeps the faster tile size
 * and records the marginal cost per block (the slope in ns). Later batches of
 * this precision are cut with those tile sizes and split across CTAs by those
 * costs instead of by bytes. For the two CUDA-core forms (BF_FP32, BF_FP32_3M)
 * it also picks that form's CTAs per SM (up to as many as fit at once).
 * Allocates and frees its own scratch (about 240 MB) and runs on `stream`
 * (synchronised before return). Uses 80 precoder slots above the plan's
 * current slots, which it leaves unset. */
bf_status bf_autotune(bf_plan plan, bf_precision prec, void *stream);

/* The table entry used for (prec, f): marginal ns per block, tile size,
 * and whether prec has been tuned. Any output pointer may be NULL. */
bf_status bf_tune_query(bf_plan plan, bf_precision prec, int32_t f, double *ns_per_block,
                        int32_t *tile_blocks, int32_t *tuned);

/* Write / read the plan's autotune table as JSON ("libbf-tune-2"). The
 * building blocks are chosen per size and target (Sec. IV), so a table records
 * the target it was measured on: the device name, the compute capability
 * (major * 10 + minor) and the SM count. bf_tune_load refuses, with BF_EINVAL
 * and the reason in bf_last_error(plan), a table measured on another target,
 * a table without a target, and any unreadable table; the plan's table is
 * then unchanged. */
bf_status bf_tune_save(bf_plan plan, const char *path);
bf_status bf_tune_load(bf_plan plan, const char *path);

/* The target check of bf_tune_load on its own, with no plan and no CUDA call:
 * BF_OK when the table at `path` was measured on (device_name, cc, sm_count),
 * BF_EINVAL otherwise (reason in bf_last_error(NULL)). */
bf_status bf_tune_check_target(const char *path, const char *device_name, int32_t cc, int32_t sm_count);

/* Accuracy targets of bf_select_form, from the accuracy classes of the
 * reduced-precision study: BF_TARGET_FP32 (relative Frobenius error <= 1e-5)
 * is met by BF_FP32, BF_FP32_3M, BF_BF16X3 and BF_TF32X3; BF_TARGET_BF16
 * (<= 2e-2) by every form. */
typedef enum { BF_TARGET_FP32 = 0, BF_TARGET_BF16 = 1 } bf_target;

/* The optimizer's building-block choice for one batch (Sec. IV: the best
 * block per size and target). Among the forms that meet `target` and are
 * tuned on this plan (bf_autotune or bf_tune_load), returns in *prec_out the
 * one with the smallest predicted time for these groups: the sum over groups
 * of n_blocks times the measured marginal ns per block of the group's f
 * bucket, for complex64 S. *ns_out (may be NULL) receives that prediction.
 * With no tuned candidate it returns the default form (BF_BF16X3 for
 * BF_TARGET_FP32, BF_BF16 for BF_TARGET_BF16) and *ns_out = 0. Host only: no
 * CUDA call. Groups must name set precoder slots (BF_ENOTFOUND otherwise). */
bf_status bf_select_form(bf_plan plan, bf_target target, const bf_group *groups, int32_t n_groups,
                         bf_precision *prec_out, double *ns_out);

/* ------------------------------------------------------------------ accuracy report */

/* Relative Frobenius error of R against a reference, accumulated in FP64.
 *  R_dev    : n_blocks blocks of complex64 R (30,720 B each).
 *  Rref_dev : the same blocks as complex128 (FP64 pairs, 61,440 B each).
 *  per_block_dev : NULL or 2*n_blocks doubles receiving, per block,
 *                  sum |R-Rref|^2 and sum |Rref|^2.
 *  total_host    : 2 doubles receiving the totals over all blocks.
 * Synchronises `stream` (the totals are copied to the host). */
bf_status bf_errnorm(bf_plan plan, const void *R_dev, const void *Rref_dev, int64_t n_blocks,
                     double *per_block_dev, double *total_host, void *stream);

/* The same accuracy report for callers that cannot allocate device memory
 * (the paper has no counterpart; it is a library convenience). A per-TTI
 * real-time loop must not call cudaMalloc or cudaFree, which may synchronise
 * the device and take unbounded time, and some callers run where another
 * allocator owns all device memory or have no plan. This call takes no plan
 * and allocates nothing: its scratch is a fixed device array inside the
 * library, 2 doubles per block for at most BF_ERRNORM_NOALLOC_MAX_BLOCKS
 * blocks (about 1 MiB), which every GPU that loads the library keeps until
 * the process exits.
 *  R_dev, Rref_dev, n_blocks, total_host : as bf_errnorm (no per-block output).
 * n_blocks above the maximum gives BF_EINVAL (text in bf_last_error(NULL)).
 * Every call looks the array's device address up for the current device and
 * context (so a cudaDeviceReset or a change of context between calls is
 * safe); the first lookup on a device may load the library's device code, so
 * make the first call on each device before any stream capture.
 * All calls share the one array: calls whose kernels overlap on the GPU (on
 * different streams or host threads) race and may return wrong totals, so
 * order them. Synchronises `stream`. */
#define BF_ERRNORM_NOALLOC_MAX_BLOCKS 65536
bf_status bf_errnorm_noalloc(const void *R_dev, const void *Rref_dev, int64_t n_blocks,
                             double *total_host, void *stream);

/* ------------------------------------------------------------------ measurement */

/* The FP32 fused multiply-add rate of the CUDA cores of the current device,
 * the roofline denominator of the plain FP32 form: at f = 36 that form does
 * 22.4 flop per algorithmic byte, above the CUDA-core ridge, so its bound is
 * FMA issue (Sec. III: the paper's improved kernel is built on FMA). One
 * kernel of 4 CTAs of 256 threads per SM, by `mode`:
 *  0: 8 independent chains of 4 * iters scalar FMAs per thread;
 *  1: the same with packed FP32x2 FMAs (4 flop each);
 *  2: packed FP32x2 FMAs in the operand pattern of a register-blocked outer
 *     product, 16 accumulator pairs over 4 x 4 operand pairs, 16 * iters
 *     FMAs per thread. Modes 0 and 1 read one register operand per FMA (the
 *     others are kernel arguments); mode 2 reads three, two of them new, as
 *     every product loop must, so its rate is the ceiling of such a loop.
 * After one warm-up launch, the best of `reps` launches timed with CUDA
 * events on `stream` gives *tflops_host (2 flop per FMA) and *ms_host (may
 * be NULL). iters in [1, 2^24], reps in [1, 1000], mode 0..2, else
 * BF_EINVAL. Synchronises `stream`. */
bf_status bf_measure_fp32_peak(int32_t iters, int32_t reps, int32_t mode, double *tflops_host, double *ms_host,
                               void *stream);

/* Number of product kernels (or graph replays) this plan has launched so far
 * (0 for a NULL plan). */
int64_t bf_plan_launch_count(bf_plan plan);

#ifdef __cplusplus
}
#endif
#endif /* BF_H */
