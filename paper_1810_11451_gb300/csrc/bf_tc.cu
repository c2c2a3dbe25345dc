// bf_tc.cu -- tensor-core forms of R = W x S (Sec. III, beamforming equation)
// on sm_103a: tcgen05.mma with shared-memory operands (for tf32, the A operand's
// hi term in tensor memory), FP32 accumulators in tensor memory, bulk (TMA)
// copies, mbarrier pipelines.
//
// The complex product as one real GEMM, resource elements on M:
//   D[j][2i+c] = sum_kk A[j][kk] * B[kk][2i+c],  kk = 2k + c'
//   A[j][2k] = Re S[k][j],  A[j][2k+1] = Im S[k][j]                (M x K)
//   B[2k][2i] = Re W[i][k], B[2k+1][2i] = -Im W[i][k],
//   B[2k][2i+1] = Im W[i][k], B[2k+1][2i+1] = Re W[i][k]            (K x N)
// so D[j][2i] = Re R[i][j] and D[j][2i+1] = Im R[i][j]: tensor-memory lane j
// holds row j of R^T with real and imaginary parts already interleaved, and a
// warp's 32 lanes write 32 consecutive resource elements (256 contiguous
// bytes) of one antenna row of R per store. One MMA tile is M = 128 (two
// blocks of 60 resource elements, each padded to 64), N = 128 (64 antennas x
// re/im), K = 2f padded to a multiple of 16.
//
// Forms: TERMS = 1 is single pass (bf16 or fp16 operands); TERMS = 3 is the
// split form Wh*Sh + Wh*Sl + Wl*Sh with x = hi + lo, hi = bf16(x), lo =
// bf16(x - hi), or with tf32 terms (kind::tf32: 32-bit elements, K = 2f
// padded to a multiple of 8, 8 per instruction). HELD = false converts
// complex64 S on chip (raw ring -> converter warps -> operand ring); HELD =
// true bulk-loads 16-bit operand images that bf_quantize_symbols encoded
// beforehand. Every kind has the same image structure in bytes: K-major, no
// swizzle, 8-row x 16-byte core matrices 128 bytes apart along K, 8-row
// groups 8*kpad*esize bytes apart, and 32 bytes of K per instruction.
// The tf32 operands are twice as large, so the tf32 form keeps the hi term of
// S in tensor memory (A from tensor memory, one 32-bit column per K element)
// and only the lo term in shared memory: two operand stages then fit beside
// one precoder buffer and four raw slots, and conversion overlaps the MMAs.
//
// Warp roles (384 threads, one CTA per SM):
//   warp 0        bulk-loads S (raw complex64 or held images) into a ring
//   warp 1        TMEM allocation; one lane issues the MMAs and commits
//   warp 2        bulk-loads each precoder image once per run of tiles
//   warps 4..7    (complex64 input) convert raw S into the operand ring
//   warps 8..11   epilogue: tensor memory -> registers -> global R
// Tensor memory holds two or four 128-column accumulators (two for tf32,
// whose hi operand stages take the other 256 columns) so the MMAs of later
// tiles overlap the epilogue of earlier ones.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "bf_device.cuh"
#include "bf_internal.h"

namespace bfi {

// Converter and epilogue warps (the epilogue count a multiple of 4: warp w
// reads tensor-memory lanes 32*(w%4) .. 32*(w%4)+31).
#ifndef BF_TC_CONV_WARPS
#define BF_TC_CONV_WARPS 4
#endif
#ifndef BF_TC_EPI_WARPS
#define BF_TC_EPI_WARPS 4
#endif
constexpr int TC_CONV_WARPS = BF_TC_CONV_WARPS;
constexpr int TC_EPI_WARPS = BF_TC_EPI_WARPS;
static_assert(TC_CONV_WARPS % 4 == 0 && TC_EPI_WARPS % 4 == 0 && TC_EPI_WARPS <= 16, "warp counts");
constexpr int TC_CONV0 = 4;                          // first converter warp
constexpr int TC_EPI0 = TC_CONV0 + TC_CONV_WARPS;    // first epilogue warp (a multiple of 4)
constexpr int TC_THREADS = 32 * (TC_EPI0 + TC_EPI_WARPS);
// Accumulators in tensor memory (2 or 4: a power-of-two allocation). The
// split form on complex64 S measured faster with 2 (back to back over the
// full band, 31.4 against 31.8 us), the single-pass and held forms with 4.
#ifndef BF_TC_NACC
#define BF_TC_NACC 4
#endif
#ifndef BF_TC_SPLIT_C64_NACC
#define BF_TC_SPLIT_C64_NACC 2
#endif
constexpr int TC_NACC = BF_TC_NACC;
constexpr int TC_SPLIT_C64_NACC = BF_TC_SPLIT_C64_NACC;
static_assert((TC_NACC == 2 || TC_NACC == 4) && (TC_SPLIT_C64_NACC == 2 || TC_SPLIT_C64_NACC == 4),
              "tensor-memory allocation is a power of two columns");
constexpr int TC_ACC_COLS = 128; // N
constexpr int TC_RAW_SLOT = F_LIMIT * S_BYTES_PER_F;  // one complex64 block, 17,280 B
constexpr int SMEM_LIMIT = 232448;                     // 227 KB of dynamic shared memory per CTA

// Ring depths per form as three digits: W buffers, operand stages (tiles),
// raw complex64 slots (blocks). Chosen by measurement; each may be
// overridden at compile time (e.g. -DBF_TC_SPLIT_C64_STAGES=124). The split
// form on complex64 S double-buffers W (its next precoder loads while the
// current one is in use) at the price of a raw slot.
#ifndef BF_TC_SPLIT_C64_STAGES
#define BF_TC_SPLIT_C64_STAGES 223
#endif
#ifndef BF_TC_SPLIT_HELD_STAGES
#define BF_TC_SPLIT_HELD_STAGES 120
#endif
#ifndef BF_TC_SINGLE_C64_STAGES
#define BF_TC_SINGLE_C64_STAGES 253
#endif
#ifndef BF_TC_SINGLE_HELD_STAGES
#define BF_TC_SINGLE_HELD_STAGES 120
#endif
// tf32 split: one precoder buffer (73,728 B), two lo-term stages (36,864 B
// each) and four raw slots.
#ifndef BF_TC_TF32_C64_STAGES
#define BF_TC_TF32_C64_STAGES 124
#endif
struct Stages {
    int nw, na, nr;
};
constexpr Stages decode_stages(int code) { return {code / 100, (code / 10) % 10, code % 10}; }
constexpr Stages STAGES[2][2] = {
    {decode_stages(BF_TC_SINGLE_C64_STAGES), decode_stages(BF_TC_SINGLE_HELD_STAGES)},
    {decode_stages(BF_TC_SPLIT_C64_STAGES), decode_stages(BF_TC_SPLIT_HELD_STAGES)}};

// Operand kinds; the value is the format code of the instruction descriptor.
constexpr int OP_FP16 = 0, OP_BF16 = 1, OP_TF32 = 2;

template <int OPK>
struct OpKind {
    static constexpr int ES = OPK == OP_TF32 ? 4 : 2;  // bytes per element
    static constexpr int KSTEP = 32 / ES;              // K of one instruction
    __host__ __device__ static constexpr int kpad(int f) { return OPK == OP_TF32 ? kpad32_of(f) : kpad_of(f); }
    __host__ __device__ static constexpr int img(int kp) { return OPK == OP_TF32 ? tf32_img_bytes(kp) : tc_img_bytes(kp); }
    static constexpr int IMG_MAX = OPK == OP_TF32 ? TF32_IMG_MAX : TC_IMG_MAX;
};

template <int TERMS, bool HELD, int OPK>
struct TcCfg {
    static_assert(OPK != OP_TF32 || (TERMS == 3 && !HELD), "tf32 operands: split form on complex64 S only");
    static constexpr int IMG = OpKind<OPK>::IMG_MAX;
    static constexpr int A_TERMS = TERMS == 3 ? 2 : 1;  // hi (and lo) operand images
    static constexpr int W_TERMS = TERMS == 3 ? 2 : 1;
    static constexpr Stages ST =
        OPK == OP_TF32 ? decode_stages(BF_TC_TF32_C64_STAGES) : STAGES[TERMS == 3 ? 1 : 0][HELD ? 1 : 0];
    static constexpr int NW = ST.nw;
    static constexpr int NA = ST.na;
    static constexpr int NR = HELD ? 0 : ST.nr;
    // tf32: the hi term of each operand stage lives in tensor memory
    static constexpr bool A_TMEM = OPK == OP_TF32;
    static constexpr int NACC = A_TMEM ? 2 : (TERMS == 3 && !HELD ? TC_SPLIT_C64_NACC : TC_NACC);  // accumulators
    static constexpr int TMEM_A0 = NACC * TC_ACC_COLS; // first column of the hi stages (128 apart)
    static constexpr int TMEM_COLS = A_TMEM ? 512 : NACC * TC_ACC_COLS;
    static_assert(!A_TMEM || TMEM_A0 + 128 * (NA - 1) + 72 <= 512, "tensor-memory columns");
    static constexpr int W_BUF = W_TERMS * IMG;
    static constexpr int A_STAGE = (A_TMEM ? 1 : A_TERMS) * IMG;
    static constexpr int OFF_W = 0;
    static constexpr int OFF_A = OFF_W + NW * W_BUF;
    static constexpr int OFF_RAW = OFF_A + NA * A_STAGE;
    static constexpr int OFF_BAR = OFF_RAW + NR * TC_RAW_SLOT;
    // raw full/empty, a full/empty, w full/empty, acc full/empty, drain
    static constexpr int NBARS = 2 * NR + 2 * NA + 2 * NW + 2 * NACC + 1;
    static constexpr int SMEM = OFF_BAR + NBARS * 8 + 16;
    static_assert(SMEM <= SMEM_LIMIT, "ring depths exceed the shared memory of one CTA");
    static_assert(HELD || NR >= 2, "a two-block tile needs at least two raw slots");
};

__device__ __forceinline__ uint32_t pack2_bf16(float a, float b) {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t *>(&h);
}
__device__ __forceinline__ uint32_t pack2_fp16(float a, float b) {
    __half2 h = __floats2half2_rn(a, b);
    return *reinterpret_cast<uint32_t *>(&h);
}
__device__ __forceinline__ float2 unpack2_bf16(uint32_t u) {
    return make_float2(__uint_as_float(u << 16), __uint_as_float(u & 0xFFFF0000u));
}

// One element (re, im) of R in the output type: complex64, or a bf16 / fp16
// pair rounded to nearest even.
__device__ __forceinline__ void store_r(uint8_t *dst, float re, float im, int r_type) {
    if (r_type == R_C64) *reinterpret_cast<float2 *>(dst) = make_float2(re, im);
    else if (r_type == R_BF16) *reinterpret_cast<uint32_t *>(dst) = pack2_bf16(re, im);
    else *reinterpret_cast<uint32_t *>(dst) = pack2_fp16(re, im);
}

template <int TERMS, bool HELD, int OPK>
__global__ void __launch_bounds__(TC_THREADS, 1) bf_tc_kernel(KParams p) {
    using C = TcCfg<TERMS, HELD, OPK>;
    using K = OpKind<OPK>;
    extern __shared__ __align__(1024) uint8_t smem[];
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + C::OFF_BAR);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(bars + C::NBARS);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + C::NBARS) + 1;
    const uint32_t bar0 = bfd::smem_u32(bars);
    auto raw_full = [&](int s) { return bar0 + 8u * s; };
    auto raw_empty = [&](int s) { return bar0 + 8u * (C::NR + s); };
    auto a_full = [&](int s) { return bar0 + 8u * (2 * C::NR + s); };
    auto a_empty = [&](int s) { return bar0 + 8u * (2 * C::NR + C::NA + s); };
    auto w_full = [&](int s) { return bar0 + 8u * (2 * C::NR + 2 * C::NA + s); };
    auto w_empty = [&](int s) { return bar0 + 8u * (2 * C::NR + 2 * C::NA + C::NW + s); };
    auto acc_full = [&](int s) { return bar0 + 8u * (2 * C::NR + 2 * C::NA + 2 * C::NW + s); };
    auto acc_empty = [&](int s) {
        return bar0 + 8u * (2 * C::NR + 2 * C::NA + 2 * C::NW + C::NACC + s);
    };
    const uint32_t drain_bar = bar0 + 8u * (C::NBARS - 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr uint32_t IDESC =
        OPK == OP_TF32 ? bfd::idesc_tf32(128, TC_ACC_COLS) : bfd::idesc_f16(OPK == OP_BF16, 128, TC_ACC_COLS);

    if (threadIdx.x == 0) {
        for (int s = 0; s < C::NR; ++s) {
            bfd::mbar_init(raw_full(s), 1);
            bfd::mbar_init(raw_empty(s), TC_CONV_WARPS);  // every converter warp reads every slot
        }
        for (int s = 0; s < C::NA; ++s) {
            bfd::mbar_init(a_full(s), HELD ? 1 : TC_CONV_WARPS);
            bfd::mbar_init(a_empty(s), 1);
        }
        for (int s = 0; s < C::NW; ++s) {
            bfd::mbar_init(w_full(s), 1);
            bfd::mbar_init(w_empty(s), 1);
        }
        for (int s = 0; s < C::NACC; ++s) {
            bfd::mbar_init(acc_full(s), 1);
            bfd::mbar_init(acc_empty(s), TC_EPI_WARPS);
        }
        bfd::mbar_init(drain_bar, 1);
        *abort_flag = 0;
        bfd::mbar_init_fence();
    }
    if (warp == 1) {
        bfd::tmem_alloc(bfd::smem_u32(tmem_slot), C::TMEM_COLS);
        bfd::tmem_relinquish();
    }
    bfd::tc_fence_before();
    __syncthreads();
    bfd::tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    // The prologue above touched no global memory: let the next launch on the
    // stream begin its own. Then every role but the W producer waits for the
    // previous grid on the stream to finish (its R may be this grid's S, its S
    // this grid's R). The W producer reads only precoder images and the work
    // list, which no grid with early release writes: the precoder kernel
    // releases its dependents only by completing and work lists are uploaded
    // by copies, both ordered before this grid could start. So it loads its
    // first precoder while the previous grid drains. When the caller declares
    // that no product launch writes S (s_independent), only the epilogue --
    // the one role that writes global memory -- waits: S is loaded, converted
    // and multiplied while the previous grid finishes.
    bfd::grid_dep_launch();
    if (warp != 2 && !(p.s_independent && warp < TC_EPI0)) bfd::grid_dep_wait();
    const int t0 = p.cta_begin[blockIdx.x], t1 = p.cta_begin[blockIdx.x + 1];

    if (warp == 0) {
        // ---------------- S producer ----------------
        if (lane == 0) {
            int n = 0, nb = 0;  // tiles and (complex64 input) blocks issued
            bool ok = true;
            for (int t = t0; t < t1 && ok; ++t) {
                const Tile tl = p.tiles[t];
                if (tl.f == 0) continue;
                if constexpr (!HELD) {
                    // one raw slot per block: blocks of a tile land in consecutive slots
                    const uint32_t bytes = (uint32_t)(tl.f * S_BYTES_PER_F);
                    for (int b = 0; b < tl.nblk; ++b, ++nb) {
                        const int st = nb % C::NR;
                        if (!bfd::mbar_wait(raw_empty(st), ((nb / C::NR) + 1) & 1, abort_flag, p.status)) {
                            ok = false;
                            break;
                        }
                        bfd::mbar_arrive_expect_tx(raw_full(st), bytes);
                        bfd::bulk_g2s(bfd::smem_u32(smem + C::OFF_RAW + st * TC_RAW_SLOT),
                                      p.S + tl.s_off + (int64_t)b * bytes, bytes, raw_full(st));
                    }
                    if (!ok) break;
                } else {
                    const int st = n % C::NA;
                    if (!bfd::mbar_wait(a_empty(st), ((n / C::NA) + 1) & 1, abort_flag, p.status)) break;
                    const uint32_t term = 64u * kpad_of(tl.f) * 2u;  // one term of one block
                    bfd::mbar_arrive_expect_tx(a_full(st), term * C::A_TERMS * tl.nblk);
                    for (int b = 0; b < tl.nblk; ++b)
                        for (int q = 0; q < C::A_TERMS; ++q)
                            bfd::bulk_g2s(bfd::smem_u32(smem + C::OFF_A + st * C::A_STAGE + q * TC_IMG_MAX +
                                                        b * term),
                                          p.S + tl.s_off + (int64_t)b * term * C::A_TERMS + q * term, term,
                                          a_full(st));
                }
                ++n;
            }
            // drain: the last copies issued into each ring slot
            constexpr int NS = HELD ? C::NA : C::NR;
            const int issued = HELD ? n : nb;
            for (int m = issued > NS ? issued - NS : 0; m < issued; ++m)
                bfd::mbar_wait_drain(bar0 + 8u * ((HELD ? 2 * C::NR : 0) + m % NS), (m / NS) & 1,
                                     1000000000ull);
        }
    } else if (warp == 2) {
        // ---------------- W producer ----------------
        if (lane == 0) {
            int n = 0;
            for (int t = t0; t < t1; ++t) {
                const Tile tl = p.tiles[t];
                if (tl.f == 0 || !(tl.flags & TF_FIRST_OF_W)) continue;
                const int wb = n % C::NW;
                if (!bfd::mbar_wait(w_empty(wb), ((n / C::NW) + 1) & 1, abort_flag, p.status)) break;
                const uint32_t bytes = (uint32_t)(C::W_TERMS * K::img(K::kpad(tl.f)));
                bfd::mbar_arrive_expect_tx(w_full(wb), bytes);
                bfd::bulk_g2s(bfd::smem_u32(smem + C::OFF_W + wb * C::W_BUF),
                              p.w_tc + (int64_t)tl.prec * p.w_tc_stride, bytes, w_full(wb));
                ++n;
            }
            for (int m = n > C::NW ? n - C::NW : 0; m < n; ++m)
                bfd::mbar_wait_drain(w_full(m % C::NW), (m / C::NW) & 1, 1000000000ull);
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            int n = 0, nw = 0, wb = 0;
            for (int t = t0; t < t1; ++t) {
                const Tile tl = p.tiles[t];
                if (tl.f == 0) continue;
                if (tl.flags & TF_FIRST_OF_W) {
                    wb = nw % C::NW;
                    if (!bfd::mbar_wait(w_full(wb), (nw / C::NW) & 1, abort_flag, p.status)) break;
                    ++nw;
                }
                const int a = n % C::NA, d = n % C::NACC;
                if (!bfd::mbar_wait(a_full(a), (n / C::NA) & 1, abort_flag, p.status)) break;
                if (!bfd::mbar_wait(acc_empty(d), ((n / C::NACC) + 1) & 1, abort_flag, p.status)) break;
                bfd::tc_fence_after();
                const int kp = K::kpad(tl.f);
                const uint32_t sbo = 8u * K::ES * kp;  // 8-row groups
                const uint32_t a_hi = bfd::smem_u32(smem + C::OFF_A + a * C::A_STAGE);
                const uint32_t a_lo = a_hi + C::IMG;
                const uint32_t b_hi = bfd::smem_u32(smem + C::OFF_W + wb * C::W_BUF);
                const uint32_t b_lo = b_hi + (uint32_t)K::img(kp);
                const uint32_t dt = tmem_base + d * TC_ACC_COLS;
                if constexpr (C::A_TMEM) {
                    // hi term of S in tensor memory (8 columns per step), lo term in shared memory
                    const uint32_t at = tmem_base + C::TMEM_A0 + 128u * a;
                    const uint32_t a_lo_s = a_hi;  // the shared-memory stage holds the lo term only
                    for (int s = 0; s < kp / K::KSTEP; ++s) {
                        const uint32_t o = 256u * s;
                        bfd::umma_tf32_ts(dt, at + 8u * s, bfd::smem_desc(b_hi + o, 128, sbo), IDESC, s > 0 ? 1u : 0u);
                        bfd::umma_tf32_ts(dt, at + 8u * s, bfd::smem_desc(b_lo + o, 128, sbo), IDESC, 1u);
                        bfd::umma_tf32(dt, bfd::smem_desc(a_lo_s + o, 128, sbo), bfd::smem_desc(b_hi + o, 128, sbo),
                                       IDESC, 1u);
                    }
                } else {
                    for (int s = 0; s < kp / K::KSTEP; ++s) {
                        const uint32_t o = 256u * s;  // two 128-byte core matrices along K
                        bfd::umma_f16(dt, bfd::smem_desc(a_hi + o, 128, sbo), bfd::smem_desc(b_hi + o, 128, sbo),
                                      IDESC, s > 0 ? 1u : 0u);
                        if (TERMS == 3) {
                            bfd::umma_f16(dt, bfd::smem_desc(a_hi + o, 128, sbo),
                                          bfd::smem_desc(b_lo + o, 128, sbo), IDESC, 1u);
                            bfd::umma_f16(dt, bfd::smem_desc(a_lo + o, 128, sbo),
                                          bfd::smem_desc(b_hi + o, 128, sbo), IDESC, 1u);
                        }
                    }
                }
                bfd::umma_commit(a_empty(a));
                bfd::umma_commit(acc_full(d));
                if (tl.flags & TF_LAST_OF_W) bfd::umma_commit(w_empty(wb));
                ++n;
            }
            // Wait for every MMA issued by this thread before tensor memory is freed.
            bfd::umma_commit(drain_bar);
            bfd::mbar_wait_drain(drain_bar, 0, 1000000000ull);
        }
    } else if (warp >= TC_CONV0 && warp < TC_EPI0) {
        // ---------------- converters (complex64 S -> operand images) ----------------
        if constexpr (C::A_TMEM) {
            // tf32: thread -> one row of the two-block operand. A warp may
            // store only to tensor-memory lanes 32*(warp%4) .. +31, so row =
            // 32*(warp%4) + lane: block (warp%4)/2, resource element j =
            // 32*(warp%2) + lane; with more than four converter warps, warps
            // w and w+4 split the K columns. Each thread rounds its row's
            // values to hi = tf32(x) and lo = tf32(x - hi), stores hi to the
            // stage's tensor-memory columns (kk = 2k + re/im) and lo to the
            // shared-memory image. Every converter warp waits on and releases
            // both raw slots of every tile, so all move through the ring
            // together.
            const int q = warp & 3;
            const int part = (warp - TC_CONV0) >> 2;
            constexpr int NPART = TC_CONV_WARPS / 4;
            const int blk = q >> 1, j = (q & 1) * 32 + lane, row = 32 * q + lane;
            int n = 0, nb = 0;  // tiles and blocks consumed
            bool ok = true;
            for (int t = t0; t < t1 && ok; ++t) {
                const Tile tl = p.tiles[t];
                const int f = tl.f;
                if (f == 0) continue;
                const int a = n % C::NA;
                if (!bfd::mbar_wait(a_empty(a), ((n / C::NA) + 1) & 1, abort_flag, p.status)) break;
                for (int b = 0; b < tl.nblk && ok; ++b)
                    ok = bfd::mbar_wait(raw_full((nb + b) % C::NR), ((nb + b) / C::NR) & 1, abort_flag, p.status);
                if (!ok) break;
                bfd::tc_fence_after();  // the MMAs that read this stage have completed
                if (blk < tl.nblk) {     // warp-uniform
                    const uint8_t *raw = smem + C::OFF_RAW + ((nb + blk) % C::NR) * TC_RAW_SLOT + j * 8;
                    const int kp = K::kpad(f);
                    uint8_t *lo_row = smem + C::OFF_A + a * C::A_STAGE + (row >> 3) * (32 * kp) + (row & 7) * 16;
                    const uint32_t t_hi = tmem_base + ((uint32_t)(32 * q) << 16) + C::TMEM_A0 + 128u * a;
                    for (int g = part; g < kp / 8; g += NPART) {  // flows 4g .. 4g+3, columns 8g .. 8g+7
                        uint32_t h[8], l[8];
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            const int k = 4 * g + u;
                            float2 x = make_float2(0.f, 0.f);
                            if (k < f && j < B_RE) x = *reinterpret_cast<const float2 *>(raw + k * S_BYTES_PER_F);
                            h[2 * u] = bfd::tf32_rne_bits(x.x);
                            h[2 * u + 1] = bfd::tf32_rne_bits(x.y);
                            l[2 * u] = bfd::tf32_rne_bits(x.x - __uint_as_float(h[2 * u]));  // x - hi is exact
                            l[2 * u + 1] = bfd::tf32_rne_bits(x.y - __uint_as_float(h[2 * u + 1]));
                        }
                        *reinterpret_cast<uint4 *>(lo_row + (2 * g) * 128) = make_uint4(l[0], l[1], l[2], l[3]);
                        *reinterpret_cast<uint4 *>(lo_row + (2 * g + 1) * 128) = make_uint4(l[4], l[5], l[6], l[7]);
                        bfd::tmem_st8(t_hi + 8u * g, h);
                    }
                    bfd::tmem_st_wait();
                }
                bfd::tc_fence_before();
                bfd::fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0) {
                    for (int b = 0; b < tl.nblk; ++b) bfd::mbar_arrive(raw_empty((nb + b) % C::NR));
                    bfd::mbar_arrive(a_full(a));
                }
                nb += tl.nblk;
                ++n;
            }
        } else if constexpr (!HELD) {
            // thread -> (resource element j, first K chunk q0); every warp
            // converts part of every block, so all converter warps wait on and
            // release every raw slot in order. (Warps that skipped slots could
            // run a ring lap ahead, and a parity wait one phase early passes.)
            const int tid = threadIdx.x - 32 * TC_CONV0;
            const int j = tid & 63, q0 = tid >> 6;
            constexpr int QSTEP = TC_CONV_WARPS / 2;
            int n = 0, nb = 0;  // tiles and blocks consumed
            bool ok = true;
            for (int t = t0; t < t1 && ok; ++t) {
                const Tile tl = p.tiles[t];
                const int f = tl.f;
                if (f == 0) continue;
                const int a = n % C::NA;
                if (!bfd::mbar_wait(a_empty(a), ((n / C::NA) + 1) & 1, abort_flag, p.status)) break;
                for (int blk = 0; blk < tl.nblk; ++blk, ++nb) {
                    const int r = nb % C::NR;
                    if (!bfd::mbar_wait(raw_full(r), (nb / C::NR) & 1, abort_flag, p.status)) {
                        ok = false;
                        break;
                    }
                    if (j < B_RE) {
                        const uint8_t *raw = smem + C::OFF_RAW + r * TC_RAW_SLOT;
                        const int kp = kpad_of(f);
                        const int row = 64 * blk + j;
                        uint8_t *dst =
                            smem + C::OFF_A + a * C::A_STAGE + (row >> 3) * (16 * kp) + (row & 7) * 16;
                        for (int q = q0; q < kp / 8; q += QSTEP) {
                            float v[8];
#pragma unroll
                            for (int u = 0; u < 4; ++u) {
                                const int k = 4 * q + u;
                                float2 x = make_float2(0.f, 0.f);
                                if (k < f) x = *reinterpret_cast<const float2 *>(raw + k * S_BYTES_PER_F + j * 8);
                                v[2 * u] = x.x;
                                v[2 * u + 1] = x.y;
                            }
                            uint4 hi, lo;
                            uint32_t *h = &hi.x, *l = &lo.x;
#pragma unroll
                            for (int u = 0; u < 4; ++u) {
                                if (OPK == OP_BF16) {
                                    h[u] = pack2_bf16(v[2 * u], v[2 * u + 1]);
                                    if (TERMS == 3) {
                                        const float2 back = unpack2_bf16(h[u]);
                                        l[u] = pack2_bf16(v[2 * u] - back.x, v[2 * u + 1] - back.y);
                                    }
                                } else {
                                    h[u] = pack2_fp16(v[2 * u], v[2 * u + 1]);
                                }
                            }
                            *reinterpret_cast<uint4 *>(dst + q * 128) = hi;
                            if (TERMS == 3) *reinterpret_cast<uint4 *>(dst + TC_IMG_MAX + q * 128) = lo;
                        }
                    }
                    __syncwarp();
                    if (lane == 0) bfd::mbar_arrive(raw_empty(r));  // this warp is done with the slot
                }
                if (!ok) break;
                bfd::fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0) bfd::mbar_arrive(a_full(a));
                ++n;
            }
        }
    } else if (warp >= TC_EPI0) {
        // ---------------- epilogue ----------------
        const int q = warp & 3;                       // tensor-memory lane quadrant
        const int blk = q >> 1;                       // block of the tile
        const int j = (q & 1) * 32 + lane;            // resource element
        constexpr int NCH = 4 / (TC_EPI_WARPS / 4);   // 32-column chunks per warp
        const int c0 = ((warp - TC_EPI0) >> 2) * NCH; // first chunk of this warp
        int n = 0;
        const int64_t rs = p.r_row_stride;
        for (int t = t0; t < t1; ++t) {
            const Tile tl = p.tiles[t];
            const bool live = blk < tl.nblk && j < B_RE;
            // this lane's element of antenna 0; antenna i is rs bytes further
            uint8_t *rj = p.R + tl.r_off + (int64_t)blk * p.r_block_stride + (int64_t)j * p.r_esize;
            if (tl.f == 0) {
                if (live)
                    for (int i = 16 * c0; i < 16 * (c0 + NCH); ++i) store_r(rj + i * rs, 0.f, 0.f, p.r_type);
                continue;
            }
            const int d = n % C::NACC;
            if (!bfd::mbar_wait(acc_full(d), (n / C::NACC) & 1, abort_flag, p.status)) break;
            bfd::tc_fence_after();
            float scale = p.w_scale[tl.prec];
            if (HELD) scale *= p.s_scale[tl.sblk + (blk < tl.nblk ? blk : 0)];
            const uint32_t ta = tmem_base + ((uint32_t)(32 * q) << 16) + d * TC_ACC_COLS;
#pragma unroll 1
            for (int c = c0; c < c0 + NCH; ++c) {
                uint32_t v[32];
                bfd::tmem_ld32(ta + 32 * c, v);
                bfd::tmem_ld_wait();
                if (live) {
                    if (p.r_type == R_C64) {
#pragma unroll
                        for (int u = 0; u < 16; ++u)
                            *reinterpret_cast<float2 *>(rj + (16 * c + u) * rs) = make_float2(
                                __uint_as_float(v[2 * u]) * scale, __uint_as_float(v[2 * u + 1]) * scale);
                    } else {
#pragma unroll
                        for (int u = 0; u < 16; ++u)
                            store_r(rj + (16 * c + u) * rs, __uint_as_float(v[2 * u]) * scale,
                                    __uint_as_float(v[2 * u + 1]) * scale, p.r_type);
                    }
                }
            }
            bfd::tc_fence_before();
            __syncwarp();
            if (lane == 0) bfd::mbar_arrive(acc_empty(d));
            ++n;
        }
    }

    __syncthreads();
    if (warp == 1) {
        bfd::tc_fence_after();
        bfd::tmem_dealloc(tmem_base, C::TMEM_COLS);
    }
}

template <int TERMS, bool HELD, int OPK>
static cudaError_t configure_tc_t() {
    return cudaFuncSetAttribute(bf_tc_kernel<TERMS, HELD, OPK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                TcCfg<TERMS, HELD, OPK>::SMEM);
}

template <int TERMS, bool HELD, int OPK>
static cudaError_t launch_tc_t(const KParams &p, int n_cta, cudaStream_t stream) {
    // Programmatic stream serialization: this launch may begin its prologue
    // while the previous kernel on the stream finishes (see grid_dep_wait).
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(n_cta);
    cfg.blockDim = dim3(TC_THREADS);
    cfg.dynamicSmemBytes = TcCfg<TERMS, HELD, OPK>::SMEM;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, bf_tc_kernel<TERMS, HELD, OPK>, p);
}

// Raise every instance's dynamic shared-memory limit (once, before launches).
cudaError_t configure_tc() {
    cudaError_t e;
    if ((e = configure_tc_t<3, true, OP_BF16>()) != cudaSuccess) return e;
    if ((e = configure_tc_t<3, false, OP_BF16>()) != cudaSuccess) return e;
    if ((e = configure_tc_t<1, true, OP_BF16>()) != cudaSuccess) return e;
    if ((e = configure_tc_t<1, false, OP_BF16>()) != cudaSuccess) return e;
    if ((e = configure_tc_t<1, true, OP_FP16>()) != cudaSuccess) return e;
    if ((e = configure_tc_t<1, false, OP_FP16>()) != cudaSuccess) return e;
    return configure_tc_t<3, false, OP_TF32>();
}

// prec: BF_BF16, BF_FP16, BF_BF16X3 or BF_TF32X3 (complex64 S only).
cudaError_t launch_tc(int prec, bool held, const KParams &p, int n_cta, cudaStream_t stream) {
    if (prec == BF_TF32X3) return launch_tc_t<3, false, OP_TF32>(p, n_cta, stream);
    if (prec == BF_BF16X3) return held ? launch_tc_t<3, true, OP_BF16>(p, n_cta, stream)
                                       : launch_tc_t<3, false, OP_BF16>(p, n_cta, stream);
    if (prec == BF_BF16) return held ? launch_tc_t<1, true, OP_BF16>(p, n_cta, stream)
                                     : launch_tc_t<1, false, OP_BF16>(p, n_cta, stream);
    return held ? launch_tc_t<1, true, OP_FP16>(p, n_cta, stream) : launch_tc_t<1, false, OP_FP16>(p, n_cta, stream);
}

int tc_smem_bytes(int prec, bool held) {
    if (prec == BF_TF32X3) return TcCfg<3, false, OP_TF32>::SMEM;
    if (prec == BF_BF16X3) return held ? TcCfg<3, true, OP_BF16>::SMEM : TcCfg<3, false, OP_BF16>::SMEM;
    return held ? TcCfg<1, true, OP_BF16>::SMEM : TcCfg<1, false, OP_BF16>::SMEM;
}

}  // namespace bfi
