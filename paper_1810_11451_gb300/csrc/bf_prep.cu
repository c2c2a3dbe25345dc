// bf_prep.cu -- the kernels around the product: precoder images (W is
// constant across many S, Sec. III, so it is converted once), the held-S
// encoder for the tensor-core forms, and the FP64 accuracy report.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "bf_device.cuh"
#include "bf_internal.h"
#include "bf_prep.h"

namespace bfi {

// Exact 2^e as an FP32 (-149 <= e <= 127), built from the IEEE-754 fields.
__device__ __forceinline__ float pow2f_exact(int e) {
    if (e >= -126) return __uint_as_float((uint32_t)(e + 127) << 23);
    return __uint_as_float(1u << (e + 149));
}

// ceil(log2 m) for a positive finite FP32 m, read from its exponent and
// mantissa fields (exact; no math library).
__device__ __forceinline__ int ceil_log2_exact(float m) {
    const uint32_t b = __float_as_uint(m);
    const int e = (int)((b >> 23) & 0xFFu);
    const uint32_t man = b & 0x7FFFFFu;
    if (e == 0) {  // subnormal: m = man * 2^-149
        const int hb = 31 - __clz(man);
        return (man == (1u << hb)) ? hb - 149 : hb - 148;
    }
    return man == 0 ? e - 127 : e - 126;
}

// Block-wide max of non-negative floats (blockDim.x a multiple of 32, <= 1024).
__device__ float block_max(float v, float *red) {
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) red[w] = v;
    __syncthreads();
    if (w == 0) {
        v = l < (int)(blockDim.x >> 5) ? red[l] : 0.f;
        for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (l == 0) red[0] = v;
    }
    __syncthreads();
    const float r = red[0];
    __syncthreads();
    return r;
}

// Byte offset of element (row, col) in a K-major, no-swizzle tensor-core
// operand image with K = kpad columns: 8x8 tiles of 16-bit values, tiles
// along K 128 bytes apart, 8-row groups 16*kpad bytes apart.
__device__ __forceinline__ int tc_offset(int row, int col, int kpad) {
    return (row >> 3) * (16 * kpad) + (col >> 3) * 128 + (row & 7) * 16 + (col & 7) * 2;
}

// The same for 32-bit (tf32) values: 8x4 tiles, 8-row groups 32*kpad bytes apart.
__device__ __forceinline__ int tc_offset32(int row, int col, int kpad) {
    return (row >> 3) * (32 * kpad) + (col >> 2) * 128 + (row & 7) * 16 + (col & 3) * 4;
}

// ------------------------------------------------------------------ precoders
// One CTA per precoder. Writes the FP32 planar image, the bf16 hi|lo image,
// the fp16 image, the tf32 hi|lo image (all three scaled by 1/scale) and the
// scale.
__global__ void __launch_bounds__(256) bf_precoder_kernel(const float2 *__restrict__ W,
                                                          const PrecJob *__restrict__ jobs,
                                                          uint8_t *w_simt, uint8_t *w_bf16x2,
                                                          uint8_t *w_fp16, uint8_t *w_tf32x2,
                                                          float *w_scale) {
    __shared__ float red[32];
    const PrecJob jb = jobs[blockIdx.x];
    const int f = jb.f, n = N_ANT * f;
    const float2 *w = W + jb.w_off;
    float m = 0.f;
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
        const float2 v = w[e];
        m = fmaxf(m, fmaxf(fabsf(v.x), fabsf(v.y)));
    }
    m = block_max(m, red);
    const int ex = m > 0.f ? ceil_log2_exact(m) : 0;
    const float scale = pow2f_exact(ex < 127 ? ex : 127);
    const float inv = pow2f_exact(-ex > -149 ? (-ex < 127 ? -ex : 127) : -149);

    float *simt = reinterpret_cast<float *>(w_simt + (int64_t)jb.slot * W_SIMT_STRIDE);
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
        const int i = e / f, k = e - i * f;
        const float2 v = w[e];
        simt[k * N_ANT + i] = v.x;
        simt[n + k * N_ANT + i] = v.y;
        simt[2 * n + k * N_ANT + i] = v.x + v.y;
    }
    const int kpad = kpad_of(f), kpad32 = kpad32_of(f);  // kpad32 <= kpad
    uint8_t *hi = w_bf16x2 + (int64_t)jb.slot * W_BF16X2_STRIDE;
    uint8_t *lo = hi + tc_img_bytes(kpad);
    uint8_t *h16 = w_fp16 + (int64_t)jb.slot * W_FP16_STRIDE;
    uint8_t *hi32 = w_tf32x2 + (int64_t)jb.slot * W_TF32X2_STRIDE;
    uint8_t *lo32 = hi32 + tf32_img_bytes(kpad32);
    // B operand (N = 128 rows n = 2i + c, K = kpad columns kk = 2k + c'):
    // row 2i: (Re W, -Im W); row 2i+1: (Im W, Re W).
    for (int e = threadIdx.x; e < 128 * kpad; e += blockDim.x) {
        const int nrow = e / kpad, kk = e - nrow * kpad;
        const int i = nrow >> 1, c = nrow & 1, k = kk >> 1, c2 = kk & 1;
        float v = 0.f;
        if (k < f) {
            const float2 x = w[i * f + k];
            v = c == 0 ? (c2 == 0 ? x.x : -x.y) : (c2 == 0 ? x.y : x.x);
        }
        const float xs = v * inv;
        const __nv_bfloat16 bh = __float2bfloat16_rn(xs);
        const __nv_bfloat16 bl = __float2bfloat16_rn(xs - __bfloat162float(bh));
        const __half hh = __float2half_rn(xs);
        const int off = tc_offset(nrow, kk, kpad);
        *reinterpret_cast<__nv_bfloat16 *>(hi + off) = bh;
        *reinterpret_cast<__nv_bfloat16 *>(lo + off) = bl;
        *reinterpret_cast<__half *>(h16 + off) = hh;
        if (kk < kpad32) {
            const uint32_t th = bfd::tf32_rne_bits(xs);
            const int o32 = tc_offset32(nrow, kk, kpad32);
            *reinterpret_cast<uint32_t *>(hi32 + o32) = th;
            *reinterpret_cast<uint32_t *>(lo32 + o32) = bfd::tf32_rne_bits(xs - __uint_as_float(th));
        }
    }
    if (threadIdx.x == 0) w_scale[jb.slot] = scale;
}

cudaError_t launch_precoders(const float2 *W, const PrecJob *jobs, int n_jobs, uint8_t *w_simt,
                             uint8_t *w_bf16x2, uint8_t *w_fp16, uint8_t *w_tf32x2, float *w_scale,
                             cudaStream_t st) {
    if (n_jobs <= 0) return cudaSuccess;
    bf_precoder_kernel<<<n_jobs, 256, 0, st>>>(W, jobs, w_simt, w_bf16x2, w_fp16, w_tf32x2, w_scale);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ held S
// Grid (max blocks per group, n_groups); one CTA per block.
template <int FMT>  // 0 = bf16, 1 = fp16, 2 = bf16 hi|lo
__global__ void __launch_bounds__(256) bf_quantize_kernel(const uint8_t *__restrict__ S,
                                                          const QGroup *__restrict__ groups,
                                                          uint8_t *Sq, float *scale_out) {
    __shared__ float red[32];
    const QGroup g = groups[blockIdx.y];
    const int b = blockIdx.x;
    if (b >= g.nb) return;
    const int f = g.f, kpad = kpad_of(f);
    const float2 *s = reinterpret_cast<const float2 *>(S + g.s_off + (int64_t)b * f * S_BYTES_PER_F);
    // One task = one row (resource element j) and one 8-column chunk q (flows
    // 4q..4q+3): consecutive threads take consecutive rows, so the reads of a
    // warp cover 256 contiguous bytes of one flow row of S and its writes 16
    // contiguous bytes per row, 128 per 8 rows. The block is read once into
    // registers (all loads in flight together), reduced, then encoded.
    constexpr int NT = 256, MAXT = (64 * (KPAD_MAX / 8) + NT - 1) / NT;
    const int n_tasks = 64 * (kpad / 8);
    float2 v[MAXT][4];
    float m = 0.f;
#pragma unroll
    for (int i = 0; i < MAXT; ++i) {
        const int e = threadIdx.x + i * NT, q = e >> 6, row = e & 63;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int k = 4 * q + u;
            v[i][u] = (e < n_tasks && row < B_RE && k < f) ? s[k * B_RE + row] : make_float2(0.f, 0.f);
            m = fmaxf(m, fmaxf(fabsf(v[i][u].x), fabsf(v[i][u].y)));
        }
    }
    m = block_max(m, red);
    const int ex = m > 0.f ? ceil_log2_exact(m) : 0;
    const float scale = pow2f_exact(ex < 127 ? ex : 127);
    const float inv = pow2f_exact(-ex > -149 ? (-ex < 127 ? -ex : 127) : -149);
    constexpr int TERMS = FMT == 2 ? 2 : 1;
    uint8_t *dst = Sq + g.q_off + (int64_t)b * held_block_bytes(f, TERMS);
    const int term_bytes = 64 * kpad * 2;
#pragma unroll
    for (int i = 0; i < MAXT; ++i) {
        const int e = threadIdx.x + i * NT, q = e >> 6, row = e & 63;
        if (e >= n_tasks) break;
        uint32_t hi[4], lo[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const float xr = v[i][u].x * inv, xi = v[i][u].y * inv;
            if (FMT == 1) {
                const __half2 h = __floats2half2_rn(xr, xi);
                hi[u] = *reinterpret_cast<const uint32_t *>(&h);
            } else {
                const __nv_bfloat162 h = __floats2bfloat162_rn(xr, xi);
                hi[u] = *reinterpret_cast<const uint32_t *>(&h);
                if (FMT == 2) {
                    const float2 hb = __bfloat1622float2(h);
                    const __nv_bfloat162 l = __floats2bfloat162_rn(xr - hb.x, xi - hb.y);
                    lo[u] = *reinterpret_cast<const uint32_t *>(&l);
                }
            }
        }
        const int off = tc_offset(row, 8 * q, kpad);
        *reinterpret_cast<uint4 *>(dst + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
        if (FMT == 2) *reinterpret_cast<uint4 *>(dst + term_bytes + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
    }
    if (threadIdx.x == 0) scale_out[g.blk0 + b] = scale;
}

cudaError_t launch_quantize(int prec, const uint8_t *S, const QGroup *groups, int n_groups, int max_nb,
                            uint8_t *Sq, float *scale_out, cudaStream_t st) {
    if (n_groups <= 0 || max_nb <= 0) return cudaSuccess;
    const dim3 grid(max_nb, n_groups);
    if (prec == BF_BF16) bf_quantize_kernel<0><<<grid, 256, 0, st>>>(S, groups, Sq, scale_out);
    else if (prec == BF_FP16) bf_quantize_kernel<1><<<grid, 256, 0, st>>>(S, groups, Sq, scale_out);
    else bf_quantize_kernel<2><<<grid, 256, 0, st>>>(S, groups, Sq, scale_out);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ accuracy report
__device__ double block_sum(double v, double *red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) red[w] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) r += red[i];
    __syncthreads();
    return r;  // valid in thread 0
}

// Per block: sum |R - Rref|^2 and sum |Rref|^2 in FP64 (fixed order).
__global__ void __launch_bounds__(256) bf_errnorm_kernel(const float2 *__restrict__ R,
                                                         const double2 *__restrict__ Rref,
                                                         int64_t n_blocks, double *per_block) {
    __shared__ double red[32];
    constexpr int E = N_ANT * B_RE;
    for (int64_t b = blockIdx.x; b < n_blocks; b += gridDim.x) {
        double num = 0.0, den = 0.0;
        for (int e = threadIdx.x; e < E; e += blockDim.x) {
            const float2 r = R[b * E + e];
            const double2 q = Rref[b * E + e];
            const double dr = (double)r.x - q.x, di = (double)r.y - q.y;
            num += dr * dr + di * di;
            den += q.x * q.x + q.y * q.y;
        }
        num = block_sum(num, red);
        den = block_sum(den, red);
        if (threadIdx.x == 0) {
            per_block[2 * b] = num;
            per_block[2 * b + 1] = den;
        }
    }
}

// Totals of the per-block pairs, one CTA, fixed summation order.
__global__ void __launch_bounds__(256) bf_sum_pairs_kernel(const double *__restrict__ per_block,
                                                           int64_t n, double *out) {
    __shared__ double red[32];
    double num = 0.0, den = 0.0;
    for (int64_t b = threadIdx.x; b < n; b += blockDim.x) {
        num += per_block[2 * b];
        den += per_block[2 * b + 1];
    }
    num = block_sum(num, red);
    den = block_sum(den, red);
    if (threadIdx.x == 0) {
        out[0] = num;
        out[1] = den;
    }
}

// ------------------------------------------------------------------ bounded-wait self-test
// Two roles wait on mbarriers that nothing completes, through the product
// kernels' bounded wait: thread 0 gives up at the limit and raises the abort
// flag; thread 32 starts 1 s later and leaves through the flag. out: gave up,
// its wait (ms), left early, its wait (ms).
__global__ void bf_selftest_wait_kernel(int *status, int *out) {
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ int abort_word;
    volatile int *abort_flag = &abort_word;
    if (threadIdx.x == 0) {
        bfd::mbar_init(bfd::smem_u32(&bar[0]), 1);
        bfd::mbar_init(bfd::smem_u32(&bar[1]), 1);
        *abort_flag = 0;
        bfd::mbar_init_fence();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned long long t0 = bfd::globaltimer();
        const bool ok = bfd::mbar_wait(bfd::smem_u32(&bar[0]), 0, abort_flag, status);
        out[0] = ok ? 0 : 1;
        out[1] = (int)((bfd::globaltimer() - t0) / 1000000ull);
    } else if (threadIdx.x == 32) {
        const unsigned long long d0 = bfd::globaltimer();
        while (bfd::globaltimer() - d0 < bfd::WAIT_LIMIT_NS / 2) {
        }
        const unsigned long long t0 = bfd::globaltimer();
        const bool ok = bfd::mbar_wait(bfd::smem_u32(&bar[1]), 0, abort_flag, status);
        out[2] = ok ? 0 : 1;
        out[3] = (int)((bfd::globaltimer() - t0) / 1000000ull);
    }
}

cudaError_t launch_selftest_wait(int *status, int *out, cudaStream_t st) {
    bf_selftest_wait_kernel<<<1, 64, 0, st>>>(status, out);
    return cudaGetLastError();
}

cudaError_t launch_errnorm(const float2 *R, const double2 *Rref, int64_t n_blocks, double *per_block,
                           double *total, int grid, cudaStream_t st) {
    if (n_blocks > 0) {
        const int g = (int)(n_blocks < grid ? n_blocks : grid);
        bf_errnorm_kernel<<<g, 256, 0, st>>>(R, Rref, n_blocks, per_block);
    }
    bf_sum_pairs_kernel<<<1, 256, 0, st>>>(per_block, n_blocks, total);
    return cudaGetLastError();
}

}  // namespace bfi
