// bf_internal.h -- shapes, the work-list tile and kernel parameters shared by
// the host side of libbf and its kernels.
#pragma once
#include <cstdint>

#include "bf.h"

namespace bfi {

constexpr int N_ANT = 64;    // antennas: rows of W and of R (Sec. II)
constexpr int B_RE = 60;     // resource elements: columns of S and R (Sec. III)
constexpr int F_LIMIT = 36;  // largest number of flows (Sec. III)

constexpr int S_BYTES_PER_F = B_RE * 8;          // one flow row of S, complex64: 480 B
constexpr int R_BLOCK_BYTES = N_ANT * B_RE * 8;  // one R block, complex64: 30,720 B

// Tensor-core operands: K = 2f real columns rounded up to the MMA's K step.
__host__ __device__ constexpr int kpad_of(int f) { return ((2 * f + 15) / 16) * 16; }
constexpr int KPAD_MAX = kpad_of(F_LIMIT);  // 80

// Bytes of one term of a 128-row bf16/fp16 operand image (a precoder image,
// or the two-block symbol operand of one tile).
__host__ __device__ constexpr int tc_img_bytes(int kpad) { return 128 * kpad * 2; }
constexpr int TC_IMG_MAX = tc_img_bytes(KPAD_MAX);  // 20,480

// Held S block: 64 rows x kpad columns of 16-bit values per term.
__host__ __device__ constexpr int64_t held_block_bytes(int f, int terms) {
    return (int64_t)terms * 64 * kpad_of(f) * 2;
}

// TF32 operands (BF_TF32X3): K = 2f rounded up to the MMA's K step of 8, and
// 32-bit elements; same 128-row K-major image structure as the 16-bit kinds.
__host__ __device__ constexpr int kpad32_of(int f) { return ((2 * f + 7) / 8) * 8; }
__host__ __device__ constexpr int tf32_img_bytes(int kpad) { return 128 * kpad * 4; }
constexpr int TF32_IMG_MAX = tf32_img_bytes(kpad32_of(F_LIMIT));  // 36,864

// Precisions: the four tensor-core / CUDA-core forms, the three-product
// CUDA-core form (BF_FP32_3M) and the TF32 split form (BF_TF32X3).
constexpr int N_PREC = 6;
__host__ __device__ constexpr bool simt_form(int prec) { return prec == BF_FP32 || prec == BF_FP32_3M; }
// Forms that take held (pre-encoded 16-bit) S.
__host__ __device__ constexpr bool held_form(int prec) {
    return prec == BF_BF16 || prec == BF_FP16 || prec == BF_BF16X3;
}

// FP32 precoder image for the CUDA-core kernels: planar, flow-major,
// Re W[i][k] at float index k*64 + i, Im W[i][k] at f*64 + k*64 + i, and
// Re W + Im W (rounded to FP32) at 2*f*64 + k*64 + i for the three-product form.
__host__ __device__ constexpr int simt_img_bytes(int f, int planes = 2) { return planes * N_ANT * f * 4; }
constexpr int SIMT_IMG_MAX = simt_img_bytes(F_LIMIT);      // 18,432
constexpr int SIMT3_IMG_MAX = simt_img_bytes(F_LIMIT, 3);  // 27,648

// Per-slot strides of the precoder store.
constexpr int64_t W_SIMT_STRIDE = SIMT3_IMG_MAX;
constexpr int64_t W_BF16X2_STRIDE = 2 * TC_IMG_MAX;  // hi image then lo image, compact
constexpr int64_t W_FP16_STRIDE = TC_IMG_MAX;
constexpr int64_t W_TF32X2_STRIDE = 2 * TF32_IMG_MAX;  // tf32 hi image then lo image, compact

// One work item: up to two consecutive blocks of one group (same precoder).
struct Tile {
    int64_t s_off;  // byte offset of the first block in the S buffer
    int64_t r_off;  // byte offset of the first block in the R buffer
    int32_t prec;   // precoder slot
    int32_t sblk;   // index of the first block in group order (held-S scale index)
    int16_t f;      // flows
    int16_t nblk;   // 1 or 2
    int32_t flags;  // TF_* bits, set by the host scheduler
};

// Tile flags, within one CTA's run of tiles and counting only tiles with f > 0.
constexpr int TF_FIRST_OF_W = 1;  // first tile that uses its precoder
constexpr int TF_LAST_OF_W = 2;   // last tile that uses its precoder
static_assert(sizeof(Tile) == 32, "Tile is 32 bytes");

// Kernel arguments (all pointers are device pointers).
struct KParams {
    const Tile *tiles;
    const int32_t *cta_begin;  // n_cta + 1 entries: CTA c runs tiles [cta_begin[c], cta_begin[c+1])
    const uint8_t *S;
    uint8_t *R;
    const float *s_scale;      // per block (held S), else nullptr
    const uint8_t *w_simt;     // FP32 planar images, stride W_SIMT_STRIDE
    const uint8_t *w_tc;       // bf16 hi|lo, fp16 or tf32 hi|lo images
    int64_t w_tc_stride;
    const float *w_scale;      // per slot: power of two undoing the image scale
    int *status;               // device status word
    // Output layout: element (block, antenna i, resource element j) of R at
    // tile.r_off + b*r_block_stride + i*r_row_stride + j*esize, esize 8 for
    // complex64 and 4 for the 16-bit pairs (r_type 1 = bf16, 2 = fp16).
    int64_t r_row_stride;
    int64_t r_block_stride;
    int32_t r_type;
    int32_t r_esize;
    // 1: no launch of this library (product or filter) enqueued since the
    // stream's last other operation writes S or s_scale, so the kernel reads S
    // before the previous grid on the stream completes (only its R stores wait)
    int32_t s_independent;
    int32_t reserved;
};

constexpr int R_C64 = 0, R_BF16 = 1, R_FP16 = 2;

}  // namespace bfi
