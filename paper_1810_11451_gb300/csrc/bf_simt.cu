// bf_simt.cu -- plain FP32 form of R = W x S on the CUDA cores (Sec. III,
// beamforming equation). Each complex multiply-add is four FP32 fused
// multiply-adds; no operand is reordered or shuffled in the inner loop (the
// paper's three inefficiencies of the original code -- extra flops, no FMA,
// many permutations -- do not arise).
//
// Persistent CTA over a cost-balanced run of tiles. One producer warp streams
// each block of S (480*f contiguous bytes) into a shared-memory ring with bulk
// copies and loads each precoder image once per run of tiles that share it
// (W is constant across many S, Sec. III), double-buffered so the next W
// arrives while the current one is in use. Eight compute warps each own 8
// antennas (rows of R); lane l owns resource elements 2l and 2l+1 (lanes 30
// and 31 idle). Per flow k a lane reads its two S values with one 16-byte
// shared load and the warp's 8+8 W values as broadcasts, then issues 64 FFMA.
// R rows are written with 16-byte stores, 480 contiguous bytes per warp
// (8-byte stores for 16-bit R types; rows and blocks at the layout's strides).
// The kernel is templated on the three-product form (BF_FP32_3M), which keeps
// three sums per output element and reads a third precoder plane.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "bf_device.cuh"
#include "bf_internal.h"

namespace bfi {

// Two consecutive elements of one antenna row of R in the output type:
// complex64 (16 bytes) or bf16 / fp16 pairs rounded to nearest even (8 bytes).
__device__ __forceinline__ void store_r2(uint8_t *dst, float re0, float im0, float re1, float im1, int r_type) {
    if (r_type == R_C64) {
        *reinterpret_cast<float4 *>(dst) = make_float4(re0, im0, re1, im1);
    } else if (r_type == R_BF16) {
        __nv_bfloat162 a = __floats2bfloat162_rn(re0, im0), b = __floats2bfloat162_rn(re1, im1);
        *reinterpret_cast<uint2 *>(dst) =
            make_uint2(*reinterpret_cast<uint32_t *>(&a), *reinterpret_cast<uint32_t *>(&b));
    } else {
        __half2 a = __floats2half2_rn(re0, im0), b = __floats2half2_rn(re1, im1);
        *reinterpret_cast<uint2 *>(dst) =
            make_uint2(*reinterpret_cast<uint32_t *>(&a), *reinterpret_cast<uint32_t *>(&b));
    }
}

// Antennas per compute warp (8 or 16) and S ring stages; compile-time knobs.
#ifndef BF_SIMT_RPW
#define BF_SIMT_RPW 8
#endif
#ifndef BF_SIMT_NS
#define BF_SIMT_NS 3
#endif
// Unroll of the loop over flows, per form (compile-time knobs). Measured on
// the full band: the plain form 97.0 / 87.6 / 88.8 us with 1 / 2 / 4, the
// three-product form 83.7 / 91.1 / 86.4 us.
#ifndef BF_SIMT_KUNROLL
#define BF_SIMT_KUNROLL 2
#endif
#ifndef BF_SIMT_KUNROLL_3M
#define BF_SIMT_KUNROLL_3M 1
#endif
constexpr int SIMT_KUNROLL = BF_SIMT_KUNROLL;
constexpr int SIMT_KUNROLL_3M = BF_SIMT_KUNROLL_3M;
constexpr int SIMT_RPW = BF_SIMT_RPW;
static_assert(SIMT_RPW == 8 || SIMT_RPW == 16, "rows per warp");
constexpr int SIMT_CWARPS = N_ANT / SIMT_RPW;          // compute warps
constexpr int SIMT_THREADS = (SIMT_CWARPS + 1) * 32;   // + one producer warp
#ifndef BF_SIMT_MIN_CTAS
#define BF_SIMT_MIN_CTAS (SIMT_RPW == 8 ? 2 : 3)
#endif
constexpr int SIMT_MIN_CTAS = BF_SIMT_MIN_CTAS;        // resident CTAs per SM the registers allow
constexpr int SIMT_NS = BF_SIMT_NS;                    // S ring stages
constexpr int SIMT_NW = 2;                             // W buffers
constexpr int SIMT_S_STAGE = F_LIMIT * S_BYTES_PER_F;  // 17,280 B
constexpr int SIMT_NBARS = 2 * SIMT_NS + 2 * SIMT_NW;
// Shared-memory layout: W buffers (2 planes, or 3 for the three-product
// form) | S ring | barriers.
template <bool G3M>
struct SimtCfg {
    static constexpr int W_BUF = G3M ? SIMT3_IMG_MAX : SIMT_IMG_MAX;
    static constexpr int OFF_S = SIMT_NW * W_BUF;
    static constexpr int OFF_BAR = OFF_S + SIMT_NS * SIMT_S_STAGE;
    static constexpr int SMEM = OFF_BAR + SIMT_NBARS * 8 + 16;
};

// G3M: the three-product form (BF_FP32_3M). Per antenna and resource element
// it keeps P1 = sum Wr Sr, P2 = sum Wi Si and P3 = sum (Wr + Wi)(Sr + Si), 3
// FFMA per complex multiply-add instead of 4, and writes Re = P1 - P2,
// Im = (P3 - P1) - P2. Wr + Wi comes from the image's third plane (loading it
// measured faster than adding the two planes in registers: 93.6 vs 98.3 us
// on the full band); the form is still slower than the plain one (87.9 us):
// this kernel is not bound by its FFMA count.
template <bool G3M>
__global__ void __launch_bounds__(SIMT_THREADS, SIMT_MIN_CTAS) bf_simt_kernel(KParams p) {
    using C = SimtCfg<G3M>;
    extern __shared__ __align__(1024) uint8_t smem[];
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + C::OFF_BAR);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(bars + SIMT_NBARS);
    const uint32_t bar0 = bfd::smem_u32(bars);
    auto s_full = [&](int s) { return bar0 + 8u * s; };
    auto s_empty = [&](int s) { return bar0 + 8u * (SIMT_NS + s); };
    auto w_full = [&](int w) { return bar0 + 8u * (2 * SIMT_NS + w); };
    auto w_empty = [&](int w) { return bar0 + 8u * (2 * SIMT_NS + SIMT_NW + w); };

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < SIMT_NS; ++s) {
            bfd::mbar_init(s_full(s), 1);
            bfd::mbar_init(s_empty(s), SIMT_CWARPS);
        }
        for (int w = 0; w < SIMT_NW; ++w) {
            bfd::mbar_init(w_full(w), 1);
            bfd::mbar_init(w_empty(w), SIMT_CWARPS);
        }
        *abort_flag = 0;
        bfd::mbar_init_fence();
    }
    __syncthreads();
    // No global memory touched yet: let the next launch start its prologue.
    // The previous kernel on the stream may still run. The producer waits for
    // it just before its first S copy (not at all when the caller declares S
    // independent of pending product launches), so its first precoder image
    // loads while the previous grid drains (precoder images and work lists are
    // never written by a grid with early release: both are complete before
    // this grid can start). The compute warps read only shared memory and the
    // work list: with independent S they start computing at once and wait
    // just before their first store of R; otherwise they have nothing to do
    // before S arrives and wait here, blocked rather than polling the S ring
    // beside the previous grid's CTA on the same SM.
    bfd::grid_dep_launch();
    if (warp != SIMT_CWARPS && !p.s_independent) bfd::grid_dep_wait();
    const int t0 = p.cta_begin[blockIdx.x], t1 = p.cta_begin[blockIdx.x + 1];

    if (warp == SIMT_CWARPS) {
        // ---------------- producer ----------------
        if (lane == 0) {
            int nS = 0, nW = 0;
            bool ok = true, dep_done = false;
            for (int t = t0; t < t1 && ok; ++t) {
                const Tile tl = p.tiles[t];
                if (tl.f == 0) continue;
                if (tl.flags & TF_FIRST_OF_W) {
                    const int wb = nW % SIMT_NW;
                    if (!bfd::mbar_wait(w_empty(wb), ((nW / SIMT_NW) + 1) & 1, abort_flag, p.status)) {
                        ok = false;
                        break;
                    }
                    const uint32_t bytes = (uint32_t)simt_img_bytes(tl.f, G3M ? 3 : 2);
                    bfd::mbar_arrive_expect_tx(w_full(wb), bytes);
                    bfd::bulk_g2s(bfd::smem_u32(smem + wb * C::W_BUF),
                                  p.w_simt + (int64_t)tl.prec * W_SIMT_STRIDE, bytes, w_full(wb));
                    ++nW;
                }
                if (!dep_done) {
                    if (!p.s_independent) bfd::grid_dep_wait();
                    dep_done = true;
                }
                const uint32_t bytes = (uint32_t)(tl.f * S_BYTES_PER_F);
                for (int b = 0; b < tl.nblk; ++b) {
                    const int st = nS % SIMT_NS;
                    if (!bfd::mbar_wait(s_empty(st), ((nS / SIMT_NS) + 1) & 1, abort_flag, p.status)) {
                        ok = false;
                        break;
                    }
                    bfd::mbar_arrive_expect_tx(s_full(st), bytes);
                    bfd::bulk_g2s(bfd::smem_u32(smem + C::OFF_S + st * SIMT_S_STAGE),
                                  p.S + tl.s_off + (int64_t)b * bytes, bytes, s_full(st));
                    ++nS;
                }
            }
            // Never leave the CTA while one of its bulk copies may still be
            // writing shared memory (only possible after an abort).
            for (int n = nS > SIMT_NS ? nS - SIMT_NS : 0; n < nS; ++n)
                bfd::mbar_wait_drain(s_full(n % SIMT_NS), (n / SIMT_NS) & 1, 1000000000ull);
            for (int n = nW > SIMT_NW ? nW - SIMT_NW : 0; n < nW; ++n)
                bfd::mbar_wait_drain(w_full(n % SIMT_NW), (n / SIMT_NW) & 1, 1000000000ull);
        }
    } else {
        // ---------------- compute warps ----------------
        const int i0 = warp * SIMT_RPW;     // first antenna of this warp
        const int jl = lane < 30 ? lane : 29;  // lanes 30, 31 mirror lane 29 and store nothing
        int nS = 0, nW = 0, wb = 0;
        bool ok = true, dep_done = false;
        auto before_store = [&] {
            if (!dep_done) {
                bfd::grid_dep_wait();
                dep_done = true;
            }
        };
        for (int t = t0; t < t1 && ok; ++t) {
            const Tile tl = p.tiles[t];
            const int f = tl.f;
            if (f == 0) {
                // empty sum: R = 0
                before_store();
                if (lane < 30) {
                    for (int b = 0; b < tl.nblk; ++b) {
                        uint8_t *rb = p.R + tl.r_off + (int64_t)b * p.r_block_stride;
#pragma unroll
                        for (int r = 0; r < SIMT_RPW; ++r)
                            store_r2(rb + (i0 + r) * p.r_row_stride + lane * 2 * p.r_esize, 0.f, 0.f, 0.f, 0.f,
                                     p.r_type);
                    }
                }
                continue;
            }
            if (tl.flags & TF_FIRST_OF_W) {
                wb = nW % SIMT_NW;
                if (!bfd::mbar_wait(w_full(wb), (nW / SIMT_NW) & 1, abort_flag, p.status)) {
                    ok = false;
                    break;
                }
                ++nW;
            }
            const float *Wr = reinterpret_cast<const float *>(smem + wb * C::W_BUF);
            const float *Wi = Wr + f * N_ANT;
            const float *Ws = Wi + f * N_ANT;  // Wr + Wi (three-product form)
            for (int b = 0; b < tl.nblk; ++b) {
                const int st = nS % SIMT_NS;
                if (!bfd::mbar_wait(s_full(st), (nS / SIMT_NS) & 1, abort_flag, p.status)) {
                    ok = false;
                    break;
                }
                const float *Sb = reinterpret_cast<const float *>(smem + C::OFF_S + st * SIMT_S_STAGE);
                float ar[SIMT_RPW][2], ai[SIMT_RPW][2];
#pragma unroll
                for (int r = 0; r < SIMT_RPW; ++r) ar[r][0] = ar[r][1] = ai[r][0] = ai[r][1] = 0.f;
                if constexpr (G3M) {
                    float p3[SIMT_RPW][2];  // ar holds P1, ai holds P2
#pragma unroll
                    for (int r = 0; r < SIMT_RPW; ++r) p3[r][0] = p3[r][1] = 0.f;
#pragma unroll SIMT_KUNROLL_3M
                    for (int k = 0; k < f; ++k) {
                        const float4 s = *reinterpret_cast<const float4 *>(Sb + k * (2 * B_RE) + 4 * jl);
                        const float s0 = s.x + s.y, s1 = s.z + s.w;
#pragma unroll
                        for (int q = 0; q < SIMT_RPW / 4; ++q) {
                            const float4 w = *reinterpret_cast<const float4 *>(Wr + k * N_ANT + i0 + 4 * q);
                            const float4 v = *reinterpret_cast<const float4 *>(Wi + k * N_ANT + i0 + 4 * q);
                            const float4 u = *reinterpret_cast<const float4 *>(Ws + k * N_ANT + i0 + 4 * q);
                            const float wr4[4] = {w.x, w.y, w.z, w.w}, wi4[4] = {v.x, v.y, v.z, v.w},
                                        ws4[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
                            for (int e = 0; e < 4; ++e) {
                                const int r = 4 * q + e;
                                ar[r][0] = fmaf(wr4[e], s.x, ar[r][0]);
                                ai[r][0] = fmaf(wi4[e], s.y, ai[r][0]);
                                p3[r][0] = fmaf(ws4[e], s0, p3[r][0]);
                                ar[r][1] = fmaf(wr4[e], s.z, ar[r][1]);
                                ai[r][1] = fmaf(wi4[e], s.w, ai[r][1]);
                                p3[r][1] = fmaf(ws4[e], s1, p3[r][1]);
                            }
                        }
                    }
#pragma unroll
                    for (int r = 0; r < SIMT_RPW; ++r)
#pragma unroll
                        for (int c = 0; c < 2; ++c) {
                            const float p1 = ar[r][c], p2 = ai[r][c];
                            ar[r][c] = p1 - p2;
                            ai[r][c] = (p3[r][c] - p1) - p2;
                        }
                } else {
#pragma unroll SIMT_KUNROLL
                for (int k = 0; k < f; ++k) {
                    const float4 s = *reinterpret_cast<const float4 *>(Sb + k * (2 * B_RE) + 4 * jl);
                    float wr[SIMT_RPW], wi[SIMT_RPW];
#pragma unroll
                    for (int q = 0; q < SIMT_RPW / 4; ++q) {  // broadcast loads of the warp's antennas
                        const float4 w = *reinterpret_cast<const float4 *>(Wr + k * N_ANT + i0 + 4 * q);
                        const float4 v = *reinterpret_cast<const float4 *>(Wi + k * N_ANT + i0 + 4 * q);
                        wr[4 * q] = w.x, wr[4 * q + 1] = w.y, wr[4 * q + 2] = w.z, wr[4 * q + 3] = w.w;
                        wi[4 * q] = v.x, wi[4 * q + 1] = v.y, wi[4 * q + 2] = v.z, wi[4 * q + 3] = v.w;
                    }
#pragma unroll
                    for (int r = 0; r < SIMT_RPW; ++r) {
                        ar[r][0] = fmaf(wr[r], s.x, ar[r][0]);
                        ar[r][0] = fmaf(-wi[r], s.y, ar[r][0]);
                        ai[r][0] = fmaf(wr[r], s.y, ai[r][0]);
                        ai[r][0] = fmaf(wi[r], s.x, ai[r][0]);
                        ar[r][1] = fmaf(wr[r], s.z, ar[r][1]);
                        ar[r][1] = fmaf(-wi[r], s.w, ar[r][1]);
                        ai[r][1] = fmaf(wr[r], s.w, ai[r][1]);
                        ai[r][1] = fmaf(wi[r], s.z, ai[r][1]);
                    }
                }
                }
                __syncwarp();
                if (lane == 0) bfd::mbar_arrive(s_empty(st));
                ++nS;
                before_store();
                if (lane < 30) {
                    uint8_t *rb = p.R + tl.r_off + (int64_t)b * p.r_block_stride;
#pragma unroll
                    for (int r = 0; r < SIMT_RPW; ++r)
                        store_r2(rb + (i0 + r) * p.r_row_stride + lane * 2 * p.r_esize, ar[r][0], ai[r][0], ar[r][1],
                                 ai[r][1], p.r_type);
                }
            }
            if (ok && (tl.flags & TF_LAST_OF_W)) {
                __syncwarp();
                if (lane == 0) bfd::mbar_arrive(w_empty(wb));
            }
        }
    }
    __syncthreads();
}

// Raise the kernel's dynamic shared-memory limit (once per process, before
// any launch or graph capture).
cudaError_t configure_simt() {
    cudaError_t e = cudaFuncSetAttribute(bf_simt_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         SimtCfg<false>::SMEM);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(bf_simt_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                SimtCfg<true>::SMEM);
}

cudaError_t launch_simt(const KParams &p, int n_cta, cudaStream_t stream, bool g3m) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(n_cta);
    cfg.blockDim = dim3(SIMT_THREADS);
    cfg.dynamicSmemBytes = g3m ? SimtCfg<true>::SMEM : SimtCfg<false>::SMEM;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;  // see grid_dep_wait
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return g3m ? cudaLaunchKernelEx(&cfg, bf_simt_kernel<true>, p) : cudaLaunchKernelEx(&cfg, bf_simt_kernel<false>, p);
}

int simt_smem_bytes() { return SimtCfg<true>::SMEM; }

// CTAs of a CUDA-core kernel that fit on one SM at once (registers, shared
// memory, threads); a launch never asks for more than this many per SM.
// g3m: the three-product form's kernel, else the plain form's.
int simt_resident_ctas(bool g3m) {
    int n = 0;
    const cudaError_t e =
        g3m ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, bf_simt_kernel<true>, SIMT_THREADS, SimtCfg<true>::SMEM)
            : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, bf_simt_kernel<false>, SIMT_THREADS,
                                                            SimtCfg<false>::SMEM);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return n > 0 ? n : 1;
}

}  // namespace bfi
