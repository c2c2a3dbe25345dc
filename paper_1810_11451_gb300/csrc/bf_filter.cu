// bf_filter.cu -- the fast-convolution filter y = IFFT(MULT(FFT(s))) of
// Sec. III (filter equation, Fig. 4), N = 2048, FP32, one fused kernel per
// call. Two kernels implement it (building blocks chosen per size and GPU by
// bf_filter_autotune, Sec. IV):
//  - bf_filter_warp_kernel (the default; see its own comment further down):
//    one warp per block of samples, two Stockham passes per transform
//    (2048 = 64 x 32), the block crossing shared memory once per transform;
//  - bf_filter_pair_kernel (see its comment): two warps per block, two
//    passes per transform (2048 = 32 x 64);
//  - bf_filter_kernel, described here: three passes per transform.
//
// Three-pass form. A team of 128 threads filters one block of 2048 samples;
// each thread holds
// 16 complex values in registers. Both transforms are Stockham passes of
// radix 16, 16 and 8 (2048 = 16 * 16 * 8): a pass reads the R values
// x[j + m N/R] of butterfly j, multiplies them by e^{-+2 pi i m k / (Ns R)},
// k = j mod Ns, takes their R-point DFT and writes them to
// (j div Ns) Ns R + k + q Ns (Ns = 1, 16, 256). The first pass reads the
// block from a shared-memory staging buffer that cp.async filled while the
// team transformed its previous block; between passes the values go through a
// padded shared-memory buffer (one pad word per 16 values keeps every access
// free of bank conflicts); the last forward pass leaves in thread t exactly
// the values X[t + 128 m], which is also what the first inverse pass needs,
// so the spectrum product happens in registers and the inverse starts there.
// The last inverse pass writes y in natural order, coalesced.
//
// The 1/N of the inverse is folded into the spectrum (a power of two, exact).
// Shared-memory bandwidth limits this kernel, so pass 2 loads only two
// twiddles per butterfly, w = e^{-2 pi i k / 256} and w^4 (k = t mod 16, at k
// and 16 + k), and forms the others by complex products of at most three
// factors. Pass 3's seven twiddles per butterfly depend only on the thread:
// each thread forms them once from w = e^{-2 pi i j / 2048} (at TW3 + j) and
// keeps them in registers for all its blocks. The tables are laid out in
// thread order, so a warp reads consecutive words.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "bf_filter.h"

namespace bff {

constexpr int N = 2048;
constexpr int TEAM = 128;                 // threads per block of samples
// Teams per CTA and CTAs per SM (compile-time knobs). 4 x 1 with the pass-3
// twiddles kept in registers measured best on the 14,336-block batch (111.4
// us; 6 x 1 without them: 113.9, with them it spills: 128.4; 5 x 1: 115.0).
#ifndef BF_FILTER_TEAMS
#define BF_FILTER_TEAMS 4
#endif
#ifndef BF_FILTER_CTAS
#define BF_FILTER_CTAS 1
#endif
// Prefetch: while a team transforms one block, cp.async copies its next
// block into a shared-memory staging buffer.
#ifndef BF_FILTER_PREFETCH
#define BF_FILTER_PREFETCH 1
#endif
constexpr int TEAMS = BF_FILTER_TEAMS;
constexpr bool PREFETCH = BF_FILTER_PREFETCH != 0;
constexpr int THREADS = TEAM * TEAMS;
constexpr int CTAS_PER_SM = BF_FILTER_CTAS;
constexpr int EBUF = N + N / 16;          // padded exchange buffer (complex values)
constexpr int TW3 = 32;                   // start of the pass-3 twiddles
constexpr int TW_SIZE = TW3 + 256;        // 288 values
constexpr int TEAM_SMEM = EBUF + (PREFETCH ? N : 0);  // exchange (+ staging) buffer per team
// shared memory: twiddles | spectrum / N | per team: exchange (+ staging)
constexpr int SMEM_BYTES = (TW_SIZE + N + TEAMS * TEAM_SMEM) * 8;
static_assert(SMEM_BYTES <= 232448, "teams per CTA exceed the shared memory of one SM");

__host__ __device__ constexpr int pad(int e) { return e + (e >> 4); }

// Complex sums as packed FP32 pairs (one instruction each on sm_100 and up):
// the butterflies are mostly additions and the kernel is issue-bound.
#ifndef BF_FILTER_PACKED
#define BF_FILTER_PACKED 1
#endif
__device__ __forceinline__ float2 cadd(float2 a, float2 b) {
#if BF_FILTER_PACKED
    return __fadd2_rn(a, b);
#else
    return make_float2(a.x + b.x, a.y + b.y);
#endif
}
__device__ __forceinline__ float2 csub(float2 a, float2 b) {
#if BF_FILTER_PACKED
    return __fadd2_rn(a, make_float2(-b.x, -b.y));
#else
    return make_float2(a.x - b.x, a.y - b.y);
#endif
}
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a times e^{DIR i theta} given w = e^{-i theta}: forward (DIR = -1) uses w,
// inverse (DIR = +1) its conjugate.
template <int DIR>
__device__ __forceinline__ float2 ctw(float2 a, float2 w) {
    if (DIR < 0) return cmul(a, w);
    return make_float2(a.x * w.x + a.y * w.y, a.y * w.x - a.x * w.y);
}
// a times DIR * i
template <int DIR>
__device__ __forceinline__ float2 cmul_i(float2 a) {
    return DIR < 0 ? make_float2(a.y, -a.x) : make_float2(-a.y, a.x);
}

// 4-point DFT in place, X_q = sum_m x_m e^{DIR 2 pi i m q / 4}.
template <int DIR>
__device__ __forceinline__ void dft4(float2 &a, float2 &b, float2 &c, float2 &d) {
    const float2 s0 = cadd(a, c), d0 = csub(a, c), s1 = cadd(b, d), d1 = cmul_i<DIR>(csub(b, d));
    a = cadd(s0, s1);
    c = csub(s0, s1);
    b = cadd(d0, d1);
    d = csub(d0, d1);
}

// cos and sin of 2 pi k / 16 for k = 1, 2, 3 (pi/8, pi/4, 3 pi/8)
constexpr float C8 = 0.923879532511286756f, S8 = 0.382683432365089772f, R2 = 0.707106781186547524f;

// e^{DIR 2 pi i k / 16} for the k = m2 * q1 products of a 4 x 4 split
template <int DIR>
__device__ __forceinline__ float2 w16(int k) {
    const float s = DIR < 0 ? -1.f : 1.f;
    switch (k) {
        case 1: return make_float2(C8, s * S8);
        case 2: return make_float2(R2, s * R2);
        case 3: return make_float2(S8, s * C8);
        case 4: return make_float2(0.f, s);
        case 6: return make_float2(-R2, s * R2);
        case 9: return make_float2(-C8, -s * S8);
        default: return make_float2(1.f, 0.f);
    }
}

// 16-point DFT: m = 4 m1 + m2, q = q1 + 4 q2; 4-point DFTs over m1, the
// twiddle e^{DIR 2 pi i m2 q1 / 16}, then 4-point DFTs over m2.
template <int DIR>
__device__ __forceinline__ void dft16(float2 (&v)[16]) {
#pragma unroll
    for (int m2 = 0; m2 < 4; ++m2) dft4<DIR>(v[m2], v[m2 + 4], v[m2 + 8], v[m2 + 12]);
    // now v[m2 + 4 q1] = U[m2][q1]
#pragma unroll
    for (int m2 = 1; m2 < 4; ++m2)
#pragma unroll
        for (int q1 = 1; q1 < 4; ++q1) v[m2 + 4 * q1] = cmul(v[m2 + 4 * q1], w16<DIR>(m2 * q1));
#pragma unroll
    for (int q1 = 0; q1 < 4; ++q1) dft4<DIR>(v[4 * q1], v[4 * q1 + 1], v[4 * q1 + 2], v[4 * q1 + 3]);
    // v[4 q1 + q2] = V[q1 + 4 q2]: transpose the 4 x 4 index grid
    float2 o[16];
#pragma unroll
    for (int q1 = 0; q1 < 4; ++q1)
#pragma unroll
        for (int q2 = 0; q2 < 4; ++q2) o[q1 + 4 * q2] = v[4 * q1 + q2];
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = o[q];
}

// 8-point DFT: m = 2 m1 + m2, q = q1 + 4 q2; 4-point DFTs over m1, the
// twiddle e^{DIR 2 pi i m2 q1 / 8}, then 2-point DFTs over m2.
template <int DIR>
__device__ __forceinline__ void dft8(float2 (&u)[8]) {
    dft4<DIR>(u[0], u[2], u[4], u[6]);
    dft4<DIR>(u[1], u[3], u[5], u[7]);
    // u[m2 + 2 q1] = U[m2][q1]
    u[3] = cmul(u[3], w16<DIR>(2));   // e^{DIR 2 pi i / 8}
    u[5] = cmul_i<DIR>(u[5]);         // e^{DIR 2 pi i 2 / 8}
    u[7] = cmul(u[7], w16<DIR>(6));   // e^{DIR 2 pi i 3 / 8}
    float2 o[8];
#pragma unroll
    for (int q1 = 0; q1 < 4; ++q1) {
        o[q1] = cadd(u[2 * q1], u[2 * q1 + 1]);
        o[q1 + 4] = csub(u[2 * q1], u[2 * q1 + 1]);
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) u[q] = o[q];
}

// The team's copy of one block (16 KB) into shared memory: 8 asynchronous
// 16-byte copies per thread, one commit group.
__device__ __forceinline__ void prefetch_block(float2 *dst, const float2 *src, int t) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    const char *g = reinterpret_cast<const char *>(src);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int off = (t + TEAM * i) * 16;
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d + off), "l"(g + off) : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}
__device__ __forceinline__ void prefetch_wait() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

__device__ __forceinline__ void team_sync(int team) {
    asm volatile("bar.sync %0, %1;" ::"r"(team + 1), "r"(TEAM) : "memory");
}

// The pass-3 twiddles of thread t, e^{-2 pi i m j / 2048} for m = 1..7 and its
// two butterflies j = t, t + 128. They depend on t only, so each thread forms
// them once (from the table's w = e^{-2 pi i j / 2048} by products) and keeps
// them in registers for every block and both transforms.
__device__ __forceinline__ void pass3_twiddles(float2 (&w3)[2][8], const float2 *tw, int t) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const float2 w1 = tw[TW3 + t + 128 * h], w2 = cmul(w1, w1), w3_ = cmul(w2, w1), w4 = cmul(w2, w2);
        w3[h][0] = make_float2(1.f, 0.f);
        w3[h][1] = w1;
        w3[h][2] = w2;
        w3[h][3] = w3_;
        w3[h][4] = w4;
        w3[h][5] = cmul(w4, w1);
        w3[h][6] = cmul(w4, w2);
        w3[h][7] = cmul(w4, w3_);
    }
}

// One transform of the block held as v[m] = x[t + 128 m] (t = thread in the
// team); leaves v[m] = X[t + 128 m]. E is the team's exchange buffer, tw the
// per-pass twiddle table, w3 the thread's pass-3 twiddles.
// With y set, pass 3 stores its outputs straight to y (element j + 256 q
// of the transform at y[j + 256 q]) as each 8-point DFT completes, instead of
// leaving them in v.
template <int DIR>
__device__ __forceinline__ void fft2048(float2 (&v)[16], float2 *E, const float2 *tw, const float2 (&w3)[2][8], int t,
                                        int team, float2 *y = nullptr) {
    // pass 1: R = 16, Ns = 1 (no twiddles)
    dft16<DIR>(v);
#pragma unroll
    for (int q = 0; q < 16; ++q) E[pad(16 * t + q)] = v[q];
    team_sync(team);
    // pass 2: R = 16, Ns = 16
#pragma unroll
    for (int m = 0; m < 16; ++m) v[m] = E[pad(t + 128 * m)];
    team_sync(team);
    {
        const int k = t & 15;
        const float2 w1 = tw[k], w4 = tw[16 + k];
        const float2 w2 = cmul(w1, w1), w3 = cmul(w2, w1);
        float2 p = w4;  // w^(4a)
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            if (a >= 2) p = cmul(p, w4);
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const int m = 4 * a + b;
                if (m == 0) continue;
                const float2 wb = b == 1 ? w1 : (b == 2 ? w2 : w3);
                const float2 w = a == 0 ? wb : (b == 0 ? p : cmul(p, wb));
                v[m] = ctw<DIR>(v[m], w);
            }
        }
    }
    dft16<DIR>(v);
    {
        const int base = 256 * (t >> 4) + (t & 15);
#pragma unroll
        for (int q = 0; q < 16; ++q) E[pad(base + 16 * q)] = v[q];
    }
    team_sync(team);
    // pass 3: R = 8, Ns = 256; butterflies j = t and j = t + 128
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int j = t + 128 * h;
        float2 u[8];
#pragma unroll
        for (int m = 0; m < 8; ++m) u[m] = E[pad(j + 256 * m)];
#pragma unroll
        for (int m = 1; m < 8; ++m) u[m] = ctw<DIR>(u[m], w3[h][m]);
        dft8<DIR>(u);
        // element j + 256 q = t + 128 (h + 2 q)
        if (y) {
#pragma unroll
            for (int q = 0; q < 8; ++q) __stcg(y + j + 256 * q, u[q]);  // L2 only
        } else {
#pragma unroll
            for (int q = 0; q < 8; ++q) v[h + 2 * q] = u[q];
        }
    }
    team_sync(team);  // the buffer is free for the next pass 1
}

// FILTER: y = IFFT(Hs * FFT(s)) with Hs = FFT(h) / N; else y = FFT(s).
// Filter launches use programmatic stream serialization: the prologue (the
// twiddle table, written at creation, and the spectrum, written by a launch
// without early release) runs while the previous launch on the stream
// finishes; s is read only after that launch completes, unless s_indep says
// that no pending launch of the library writes it, and y is always written
// after it.
template <bool FILTER>
__global__ void __launch_bounds__(THREADS, CTAS_PER_SM)
    bf_filter_kernel(const float2 *s, float2 *y, long long n_sig, const float2 *__restrict__ tw_g,
                     const float2 *__restrict__ H_g, int s_indep) {
    extern __shared__ __align__(16) float2 sm[];
    float2 *tw = sm;
    float2 *Hs = sm + TW_SIZE;
    const int team = threadIdx.x / TEAM, t = threadIdx.x % TEAM;
    float2 *E = sm + TW_SIZE + N + team * TEAM_SMEM;
    float2 *IN = E + EBUF;  // staging buffer (PREFETCH only)
    for (int i = threadIdx.x; i < N; i += THREADS) {
        if (i < TW_SIZE) tw[i] = tw_g[i];  // 288 x 8 B keeps every later region 16-byte aligned
        if (FILTER) {
            const float2 h = H_g[i];
            Hs[i] = make_float2(h.x * (1.f / N), h.y * (1.f / N));
        }
    }
    __syncthreads();
    float2 w3[2][8];
    pass3_twiddles(w3, tw, t);
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    bool dep_done = false;
    if (!s_indep) {
        asm volatile("griddepcontrol.wait;" ::: "memory");
        dep_done = true;
    }
    const long long stride = (long long)gridDim.x * TEAMS;
    long long q = (long long)blockIdx.x * TEAMS + team;
    if (PREFETCH && q < n_sig) prefetch_block(IN, s + q * N, t);
    for (; q < n_sig; q += stride) {
        float2 v[16];
        if (PREFETCH) {
            prefetch_wait();
            team_sync(team);  // every thread's copies of block q have landed
#pragma unroll
            for (int m = 0; m < 16; ++m) v[m] = IN[t + 128 * m];
            team_sync(team);  // all reads done before the next copy overwrites IN
            if (q + stride < n_sig) prefetch_block(IN, s + (q + stride) * N, t);
        } else {
            const float2 *sq = s + q * N;
#pragma unroll
            for (int m = 0; m < 16; ++m) v[m] = sq[t + 128 * m];
        }
        fft2048<-1>(v, E, tw, w3, t, team);
        float2 *yq = y + q * N;
        if (!dep_done) {
            asm volatile("griddepcontrol.wait;" ::: "memory");
            dep_done = true;
        }
        if (FILTER) {
#pragma unroll
            for (int m = 0; m < 16; ++m) v[m] = cmul(v[m], Hs[t + 128 * m]);
            fft2048<1>(v, E, tw, w3, t, team, yq);  // stores y as its last pass completes
        } else {
#pragma unroll
            for (int m = 0; m < 16; ++m) yq[t + 128 * m] = v[m];
        }
    }
}

// ---------------------------------------------------------------------------
// Two-pass form: one warp per block, 2048 = 64 x 32.
//
// Each transform is two Stockham passes instead of three, and the block
// stays in one exchange buffer E per warp (no barrier but __syncwarp):
//  - forward pass A (radix 64, Ns = 1): lane l is butterfly j = l, holds
//    x[j + 32 m], m < 64, and writes its 64-point DFT to row j of E,
//    E[64 j + q];
//  - forward pass B (radix 32, Ns = 64): butterflies j = l and l + 32, one at
//    a time, read column j, E[j + 64 m], m < 32, twist by e^{-2 pi i j m / N}
//    and give X[j + 64 q]; the product with H / N follows in registers;
//  - inverse pass B' (radix 32, Ns = 1) takes exactly those values, and its
//    output (j, q) goes back to the place it came from, E[j + 64 q], so each
//    of the two butterflies of a lane touches only its own column;
//  - inverse pass A' (radix 64, Ns = 32): butterfly j = l needs inverse
//    values (m, j), m < 64, which is row j of E, twisted by
//    e^{+2 pi i j m / N}; that twist is applied by pass B' before its store
//    (the same table values as pass B's), and pass A' stores y[j + 32 q],
//    coalesced.
// Both transforms run the forward DFT code: the inverse DFT of z is the
// conjugate of the forward DFT of conj(z). So the product writes
// conj(X H / N) (conjugation folded into the multiply), E holds conjugated
// inverse values twisted by the forward twiddles, and y is the conjugate of
// its last DFT. The 64- and 32-point DFTs run in registers as
// 8 x 8 and 8 x 4 splits with constant twiddles, each once in the code (two
// loops of two rounds), so the loop body stays small. The pass twiddles come
// from a 64 x 32 table e^{-2 pi i a b / N} (row stride 34, so a lane reads
// its row as 16-byte pairs); E has two pads
// per 64 values: the column accesses of a half-warp touch 16 distinct 8-byte
// bank pairs, and each row starts on a 16-byte boundary, so passes A and A'
// move a row as 16-byte pairs (conflict-free in 8-lane phases). The next block
// is copied into E (unpadded) with cp.async while the current one finishes
// its last pass.
constexpr int XBUF = N + N / 32;               // exchange buffer per warp (two pads per 64 values)
constexpr int TB_ROW = 34;  // even: rows start on 16-byte boundaries
constexpr int TB_SIZE = 64 * TB_ROW;           // e^{-2 pi i a b / N}, a < 64, b < 32, at a * 34 + b
// shared memory of a CTA of `warps` warps (blocks in flight), one CTA per SM;
// with hg the spectrum is read from global memory (through L1) instead of
// shared memory, which leaves room for more warps
__host__ __device__ constexpr int wsmem_bytes(int warps, bool hg = false) {
    return (TB_SIZE + (hg ? 0 : N) + warps * XBUF) * 8;
}
static_assert(wsmem_bytes(8) <= 232448, "8 warps per CTA exceed the shared memory of one SM");
static_assert(wsmem_bytes(12, true) <= 232448, "12 warps per CTA exceed the shared memory of one SM");

__host__ __device__ constexpr int padf(int e) { return e + 2 * (e >> 6); }
// Two consecutive complex values of a row of E as one 16-byte access (rows
// start on 16-byte boundaries: 66 values apart, the buffer 16-byte aligned).
__device__ __forceinline__ void store_pair(float2 *dst, float2 a, float2 b) {
    *reinterpret_cast<float4 *>(dst) = make_float4(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ void load_pair(const float2 *src, float2 &a, float2 &b) {
    const float4 t = *reinterpret_cast<const float4 *>(src);
    a = make_float2(t.x, t.y);
    b = make_float2(t.z, t.w);
}

// cos(2 pi k / 64) for k in [0, 16]
__device__ __forceinline__ float cos64(int k) {
    switch (k) {
        case 1: return 0.99518472667219693f;
        case 2: return 0.98078528040323043f;
        case 3: return 0.95694033573220882f;
        case 4: return 0.92387953251128674f;
        case 5: return 0.88192126434835505f;
        case 6: return 0.83146961230254524f;
        case 7: return 0.77301045336273699f;
        case 8: return 0.70710678118654757f;
        case 9: return 0.63439328416364549f;
        case 10: return 0.55557023301960229f;
        case 11: return 0.47139673682599781f;
        case 12: return 0.38268343236508984f;
        case 13: return 0.29028467725446233f;
        case 14: return 0.19509032201612833f;
        case 15: return 0.09801714032956077f;
        case 16: return 0.f;
        default: return 1.f;
    }
}

// a * e^{-2 pi i n / 64} for a constant n (after unrolling): quarter turns and
// odd multiples of an eighth turn take their exact short forms.
__device__ __forceinline__ float2 twc(float2 a, int n) {
    n &= 63;
    const int quad = n >> 4, k = n & 15;
    float2 r;
    if (k == 0) {
        r = a;
    } else if (k == 8) {
        r = make_float2((a.x + a.y) * R2, (a.y - a.x) * R2);
    } else {
        const float c = cos64(k), sn = cos64(16 - k);
        r = make_float2(fmaf(a.x, c, a.y * sn), fmaf(-a.x, sn, a.y * c));
    }
    if (quad == 1) return cmul_i<-1>(r);
    if (quad == 2) return make_float2(-r.x, -r.y);
    if (quad == 3) return cmul_i<1>(r);
    return r;
}

// conj(a * b) with the conjugation folded into the multiply
__device__ __forceinline__ float2 cmul_conj(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(-a.x, b.y, -a.y * b.x));
}
__device__ __forceinline__ float conj_im(float x) { return __int_as_float(__float_as_int(x) ^ 0x80000000); }

// forward 8-point DFT of v[b + s i], i < 8, in place, natural order
template <int L>
__device__ __forceinline__ void dft8_at(float2 (&v)[L], int b, int s) {
    float2 u[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) u[i] = v[b + s * i];
    dft8<-1>(u);
#pragma unroll
    for (int i = 0; i < 8; ++i) v[b + s * i] = u[i];
}

// forward 64-point DFT of v[m] (natural order) in two stages; after
// dft64_head and the eight dft8_at(v, 8 q1, 1), X[q1 + 8 q2] ends at v[8 q1 + q2]
__host__ __device__ constexpr int pos64(int q) { return 8 * (q & 7) + (q >> 3); }
// its first stage: eight 8-point DFTs and the twiddles between the stages
__device__ __forceinline__ void dft64_head(float2 (&v)[64]) {
#pragma unroll
    for (int m2 = 0; m2 < 8; ++m2) dft8_at(v, m2, 8);
#pragma unroll
    for (int m2 = 1; m2 < 8; ++m2)
#pragma unroll
        for (int q1 = 1; q1 < 8; ++q1) v[m2 + 8 * q1] = twc(v[m2 + 8 * q1], m2 * q1);
}

// forward 32-point DFT of v[m] (natural order); X[q1 + 8 q2] ends at v[4 q1 + q2]
__host__ __device__ constexpr int pos32(int q) { return 4 * (q & 7) + (q >> 3); }
// its first stage: four 8-point DFTs and the twiddles between the stages
__device__ __forceinline__ void dft32_head(float2 (&v)[32]) {
#pragma unroll
    for (int m2 = 0; m2 < 4; ++m2) dft8_at(v, m2, 4);
#pragma unroll
    for (int m2 = 1; m2 < 4; ++m2)
#pragma unroll
        for (int q1 = 1; q1 < 8; ++q1) v[m2 + 4 * q1] = twc(v[m2 + 4 * q1], 2 * m2 * q1);
}
__device__ __forceinline__ void dft32(float2 (&v)[32]) {
    dft32_head(v);
#pragma unroll
    for (int q1 = 0; q1 < 8; ++q1) dft4<-1>(v[4 * q1], v[4 * q1 + 1], v[4 * q1 + 2], v[4 * q1 + 3]);
}

// The warp's copy of one block (16 KB) into E, unpadded: 32 asynchronous
// 16-byte copies per lane, one commit group.
__device__ __forceinline__ void stage_block(float2 *dst, const float2 *src, int l) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    const char *g = reinterpret_cast<const char *>(src);
#pragma unroll
    for (int i = 0; i < 32; ++i) {
        const int off = (l + 32 * i) * 16;
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d + off), "l"(g + off) : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}

// FILTER: y = IFFT(Hs * FFT(s)) with Hs = FFT(h) / N; else y = FFT(s). The
// launch ordering is that of bf_filter_kernel (programmatic stream
// serialization; s read after the previous launch completes unless s_indep,
// y always written after it).
// HG: H / N is read from global memory (Hn_g, through L1), not shared memory.
template <bool FILTER, int WARPS, bool HG = false>
__global__ void __launch_bounds__(32 * WARPS, 1)
    bf_filter_warp_kernel(const float2 *s, float2 *y, long long n_sig, const float2 *__restrict__ tb_g,
                          const float2 *__restrict__ H_g, int s_indep, const float2 *__restrict__ Hn_g) {
    extern __shared__ __align__(16) float2 sm[];
    float2 *TB = sm;
    float2 *Hs = sm + TB_SIZE;  // H / N (not HG)
    const int warp = threadIdx.x >> 5, l = threadIdx.x & 31;
    float2 *E = sm + TB_SIZE + (HG ? 0 : N) + warp * XBUF;
    for (int i = threadIdx.x; i < (HG ? 0 : N) + TB_SIZE; i += 32 * WARPS) {
        if (i < TB_SIZE) {
            TB[i] = tb_g[i];
        } else if (FILTER) {
            const float2 h = H_g[i - TB_SIZE];
            Hs[i - TB_SIZE] = make_float2(h.x * (1.f / N), h.y * (1.f / N));
        }
    }
    __syncthreads();
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    bool dep_done = false;
    if (!s_indep) {
        asm volatile("griddepcontrol.wait;" ::: "memory");
        dep_done = true;
    }
    const long long stride = (long long)gridDim.x * WARPS;
    long long q = (long long)blockIdx.x * WARPS + warp;
    if (q < n_sig) stage_block(E, s + q * N, l);
    for (; q < n_sig; q += stride) {
        float2 v[64];
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        __syncwarp();
#pragma unroll
        for (int m = 0; m < 64; ++m) v[m] = E[l + 32 * m];
        __syncwarp();  // every lane has its inputs before E is overwritten
        // Round 0: forward pass A. Round 1: inverse pass A' (conjugated).
        float2 *yq = y + q * N;
#pragma unroll 1
        for (int round = 0;; ++round) {
            // The 64-point DFT. In the inverse round (the last) the outputs
            // of each final 8-point DFT, X[q1 + 8 q2] at v[8 q1 + q2], are
            // stored to y as soon as they are ready, which spreads the
            // block's stores over the computation (y = conj of pass A''s
            // DFT, y[l + 32 q]).
            const bool last = FILTER && round == 1;
            if (last && !dep_done) {
                asm volatile("griddepcontrol.wait;" ::: "memory");
                dep_done = true;
            }
            dft64_head(v);
#pragma unroll
            for (int q1 = 0; q1 < 8; ++q1) {
                dft8_at(v, 8 * q1, 1);
                if (last) {
#pragma unroll
                    for (int q2 = 0; q2 < 8; ++q2) {
                        const float2 r = v[8 * q1 + q2];
                        __stcg(yq + l + 32 * (q1 + 8 * q2), make_float2(r.x, conj_im(r.y)));  // L2 only
                    }
                }
            }
            if (round == 1 || !FILTER) break;
#pragma unroll
            for (int q2 = 0; q2 < 64; q2 += 2) store_pair(E + padf(64 * l + q2), v[pos64(q2)], v[pos64(q2 + 1)]);
            __syncwarp();
            // forward pass B, product, inverse pass B' for the lane's two columns
#pragma unroll 1
            for (int h = 0; h < 2; ++h) {
                const int j = l + 32 * h;
                // e^{-2 pi i j m / N}, m < 32 (table row j): pass B's twiddles,
                // and also the ones pass A' needs on this column's inverse
                // outputs (value (j, q) goes to butterfly q of pass A' as its
                // input j, twisted by e^{-2 pi i j q / N} in the conjugated
                // domain), applied by pass B' before its store so pass A'
                // reads its inputs ready. Pass B' reads them from the table
                // again: keeping them in registers (62 more) measured no faster
                // with 8 warps and made the 12-warp variant spill.
                float2 u[32];
                u[0] = E[padf(j)];
#pragma unroll
                for (int m = 0; m < 32; m += 2) {
                    float2 w0, w1;
                    load_pair(TB + j * TB_ROW + m, w0, w1);
                    if (m > 0) u[m] = cmul(E[padf(j + 64 * m)], w0);
                    u[m + 1] = cmul(E[padf(j + 64 * (m + 1))], w1);
                }
#pragma unroll 1
                for (int sub = 0;; ++sub) {
                    dft32(u);
                    if (sub == 1) break;
                    float2 t[32];
#pragma unroll
                    for (int m = 0; m < 32; ++m)
                        t[m] = cmul_conj(u[pos32(m)], HG ? __ldg(Hn_g + j + 64 * m) : Hs[j + 64 * m]);
#pragma unroll
                    for (int m = 0; m < 32; ++m) u[m] = t[m];
                }
                E[padf(j)] = u[pos32(0)];
#pragma unroll
                for (int q2 = 0; q2 < 32; q2 += 2) {
                    float2 w0, w1;
                    load_pair(TB + j * TB_ROW + q2, w0, w1);
                    if (q2 > 0) E[padf(j + 64 * q2)] = cmul(u[pos32(q2)], w0);
                    E[padf(j + 64 * (q2 + 1))] = cmul(u[pos32(q2 + 1)], w1);
                }
            }
            __syncwarp();
            // inverse pass A' input: row l of E (conjugated, already twisted)
#pragma unroll
            for (int m = 0; m < 64; m += 2) load_pair(E + padf(64 * l + m), v[m], v[m + 1]);
            __syncwarp();  // E is free: copy the next block in while this one finishes
            if (q + stride < n_sig) stage_block(E, s + (q + stride) * N, l);
        }
        if (!dep_done) {
            asm volatile("griddepcontrol.wait;" ::: "memory");
            dep_done = true;
        }
        if (!FILTER) {  // spectrum: pass B alone, X[j + 64 q]
#pragma unroll
            for (int q2 = 0; q2 < 64; q2 += 2) store_pair(E + padf(64 * l + q2), v[pos64(q2)], v[pos64(q2 + 1)]);
            __syncwarp();
#pragma unroll 1
            for (int h = 0; h < 2; ++h) {
                const int j = l + 32 * h;
                float2 u[32];
                u[0] = E[padf(j)];
#pragma unroll
                for (int m = 0; m < 32; m += 2) {
                    float2 w0, w1;
                    load_pair(TB + j * TB_ROW + m, w0, w1);
                    if (m > 0) u[m] = cmul(E[padf(j + 64 * m)], w0);
                    u[m + 1] = cmul(E[padf(j + 64 * (m + 1))], w1);
                }
                dft32(u);
#pragma unroll
                for (int q2 = 0; q2 < 32; ++q2) yq[j + 64 * q2] = u[pos32(q2)];
            }
            __syncwarp();
            if (q + stride < n_sig) stage_block(E, s + (q + stride) * N, l);
        }
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
}

// Pair form: two warps (64 lanes) per block, 32 values per lane, 2048 =
// 32 x 64. Half the registers of the one-warp form, so an SM runs 16 warps
// (four per sub-partition) instead of 8, and each block crosses shared
// memory once per transform as before:
//  - forward pass 1 (radix 32, Ns = 1): lane L = 32 w + l (w: warp of the
//    pair) is butterfly L, x[L + 64 m], m < 32, and writes E[32 L + q];
//  - forward pass 2 (radix 64, Ns = 32), split over lane pairs: butterfly
//    j = 16 w + (l & 15) belongs to lanes l < 16 (r = 0) and l + 16 (r = 1)
//    of warp w. Lane r reads the inputs m = 16 r + i and m + 32 (i < 16),
//    twisted by e^{-2 pi i j m / N} (the 64 x 32 table read transposed), and
//    takes the first radix-2 step of the 64-point DFT (decimation in
//    frequency): b = a_m + a_{m+32}, c = (a_m - a_{m+32}) e^{-2 pi i m / 64}.
//    One exchange of 16 values with the partner (shuffle, lane xor 16) gives
//    lane r = 0 all 32 b and lane r = 1 all 32 c, whose 32-point DFTs are
//    the even and odd outputs X[j + 32 k], k = 2 s + r;
//  - the product with H / N (conjugated, as in the one-warp form) in
//    registers; lanes r = 0 and 1 then hold the even and odd inputs of the
//    inverse's radix-64 butterfly j, so the inverse pass 1 starts in
//    registers with a 32-point DFT and ends with one radix-2 step
//    (decimation in time) after a second exchange, and writes E[64 j + q];
//  - inverse pass 2 (radix 32, Ns = 64): lane L reads E[L + 64 m] twisted by
//    the table and stores y[L + 64 q], coalesced.
// The exchange buffer has one pad per 32 values and one more per 512, which
// keeps every access of a half-warp free of bank conflicts in all four
// patterns. The two warps of a pair meet at a named barrier between passes;
// the next block is copied into E with cp.async while the last pass runs.
constexpr int PBUF = 2114;  // padp(N - 1) + 1
__host__ __device__ constexpr int padp(int e) { return e + (e >> 5) + (e >> 9); }
static_assert(padp(N - 1) + 1 == PBUF, "pair exchange buffer");
__host__ __device__ constexpr int psmem_bytes(int pairs) { return (TB_SIZE + N + pairs * PBUF) * 8; }
static_assert(psmem_bytes(8) <= 232448, "8 pairs per CTA exceed the shared memory of one SM");

// the two warps of pair `id` (named barrier id + 1; barrier 0 is __syncthreads)
__device__ __forceinline__ void pair_sync(int id) {
    asm volatile("bar.sync %0, 64;" ::"r"(id + 1) : "memory");
}

// The pair's copy of one block (16 KB) into E, unpadded: 16 asynchronous
// 16-byte copies per lane (L < 64), one commit group.
__device__ __forceinline__ void stage_block_pair(float2 *dst, const float2 *src, int L) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    const char *g = reinterpret_cast<const char *>(src);
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const int off = (L + 64 * i) * 16;
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d + off), "l"(g + off) : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}

// y = IFFT(Hs * FFT(s)), Hs = FFT(h) / N; launch ordering as bf_filter_kernel.
template <int PAIRS>
__global__ void __launch_bounds__(64 * PAIRS, 1)
    bf_filter_pair_kernel(const float2 *s, float2 *y, long long n_sig, const float2 *__restrict__ tb_g,
                          const float2 *__restrict__ H_g, int s_indep) {
    extern __shared__ __align__(16) float2 sm[];
    float2 *TB = sm;
    float2 *Hs = sm + TB_SIZE;
    const int warp = threadIdx.x >> 5, l = threadIdx.x & 31;
    const int pair = warp >> 1, wp = warp & 1;
    const int L = 32 * wp + l;              // passes 1 and 2': butterfly L
    const int r = l >> 4;                   // passes 2 and 1': which half of butterfly j
    const int j = 16 * wp + (l & 15);       // passes 2 and 1': butterfly j
    float2 *E = sm + TB_SIZE + N + pair * PBUF;
    for (int i = threadIdx.x; i < N + TB_SIZE; i += 64 * PAIRS) {
        if (i < TB_SIZE) {
            TB[i] = tb_g[i];
        } else {
            const float2 h = H_g[i - TB_SIZE];
            Hs[i - TB_SIZE] = make_float2(h.x * (1.f / N), h.y * (1.f / N));
        }
    }
    __syncthreads();
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    bool dep_done = false;
    if (!s_indep) {
        asm volatile("griddepcontrol.wait;" ::: "memory");
        dep_done = true;
    }
    // constant parts of the padded indices (see padp)
    const int e1 = 33 * L + (L >> 4);           // pass 1 writes E[e1 + q]
    const int e2 = j + 529 * r;                 // pass 2 reads E[e2 + 33 i] and E[e2 + 1058 + 33 i]
    const int t2 = 544 * r + j;                 // and twiddles TB[t2 + 34 i], TB[t2 + 1088 + 34 i]
    const int e3 = 66 * j + (j >> 3) + 16 * r;  // pass 1' writes E[e3 + i] and E[e3 + 33 + i]
    const int e4 = L + wp;                      // pass 2' reads E[e4 + 66 m + (m >> 3)]
    const long long stride = (long long)gridDim.x * PAIRS;
    long long q = (long long)blockIdx.x * PAIRS + pair;
    if (q < n_sig) stage_block_pair(E, s + q * N, L);
    for (; q < n_sig; q += stride) {
        float2 v[32];
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        pair_sync(pair);
#pragma unroll
        for (int m = 0; m < 32; ++m) v[m] = E[L + 64 * m];
        pair_sync(pair);  // every lane has its inputs before E is overwritten
        // forward pass 1
        dft32(v);
#pragma unroll
        for (int q2 = 0; q2 < 32; ++q2) E[e1 + q2] = v[pos32(q2)];
        pair_sync(pair);
        // forward pass 2: twist, first radix-2 step, exchange, 32-point DFT
        {
            float2 bv[16], cv[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const float2 a0 = cmul(E[e2 + 33 * i], TB[t2 + TB_ROW * i]);
                const float2 a1 = cmul(E[e2 + 1058 + 33 * i], TB[t2 + 32 * TB_ROW + TB_ROW * i]);
                bv[i] = cadd(a0, a1);
                const float2 c = twc(csub(a0, a1), i);      // e^{-2 pi i i / 64}
                cv[i] = r ? cmul_i<-1>(c) : c;              // and e^{-2 pi i 16 / 64} = -i for r = 1
            }
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const float2 snd = r ? bv[i] : cv[i];
                const float2 rcv = make_float2(__shfl_xor_sync(0xffffffffu, snd.x, 16),
                                               __shfl_xor_sync(0xffffffffu, snd.y, 16));
                v[i] = r ? rcv : bv[i];
                v[16 + i] = r ? cv[i] : rcv;
            }
        }
        dft32(v);  // X[j + 32 (2 s + r)] at v[pos32(s)]
        // product, conjugated: the inverse runs the forward DFT code
        float2 u[32];
#pragma unroll
        for (int s2 = 0; s2 < 32; ++s2) u[s2] = cmul_conj(v[pos32(s2)], Hs[j + 32 * r + 64 * s2]);
        // inverse pass 1: 32-point DFT of the even (r = 0) or odd (r = 1)
        // inputs, exchange, last radix-2 step
        dft32(u);  // G[k] at u[pos32(k)]
        pair_sync(pair);  // the partner warp has finished reading E in pass 2
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const float2 g0 = u[pos32(i)], g1 = u[pos32(16 + i)];
            const float2 snd = r ? g0 : g1;
            const float2 rcv = make_float2(__shfl_xor_sync(0xffffffffu, snd.x, 16),
                                           __shfl_xor_sync(0xffffffffu, snd.y, 16));
            const float2 P = r ? rcv : g0;
            float2 T = twc(r ? g1 : rcv, i);
            T = r ? cmul_i<-1>(T) : T;
            E[e3 + i] = cadd(P, T);
            E[e3 + 33 + i] = csub(P, T);
        }
        pair_sync(pair);
        // inverse pass 2: twist by the table, 32-point DFT, conjugate, store
        v[0] = E[e4];
#pragma unroll
        for (int m = 0; m < 32; m += 2) {
            float2 w0, w1;
            load_pair(TB + L * TB_ROW + m, w0, w1);
            if (m > 0) v[m] = cmul(E[e4 + 66 * m + (m >> 3)], w0);
            v[m + 1] = cmul(E[e4 + 66 * (m + 1) + ((m + 1) >> 3)], w1);
        }
        pair_sync(pair);  // E is free: copy the next block in while this one finishes
        if (q + stride < n_sig) stage_block_pair(E, s + (q + stride) * N, L);
        if (!dep_done) {
            asm volatile("griddepcontrol.wait;" ::: "memory");
            dep_done = true;
        }
        // the 32-point DFT, each final 4-point DFT's outputs X[q1 + 8 q2]
        // (at v[4 q1 + q2]) stored to y[L + 64 (q1 + 8 q2)] as soon as they are ready
        float2 *yq = y + q * N;
        dft32_head(v);
#pragma unroll
        for (int q1 = 0; q1 < 8; ++q1) {
            dft4<-1>(v[4 * q1], v[4 * q1 + 1], v[4 * q1 + 2], v[4 * q1 + 3]);
#pragma unroll
            for (int q2 = 0; q2 < 4; ++q2) {
                const float2 rr = v[4 * q1 + q2];
                __stcg(yq + L + 64 * (q1 + 8 * q2), make_float2(rr.x, conj_im(rr.y)));  // L2 only
            }
        }
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
}

}  // namespace bff

using namespace bff;

struct bf_filter_s {
    int device = 0, sm_count = 0;
    float2 *tw = nullptr, *H = nullptr, *hpad = nullptr;
    float2 *tb = nullptr;  // pass twiddles of the two-pass forms, e^{-2 pi i a b / N} at a * TB_ROW + b
    float2 *Hn = nullptr;  // H / N (the spectrum scaled once, for the variant that reads it from global memory)
    bool has_taps = false;
    std::string err;
    int64_t launches = 0;
    // host-buffer pipeline: copy-in, compute and copy-out streams, 3 slots
    cudaStream_t x_in = nullptr, x_run = nullptr, x_out = nullptr;
    cudaEvent_t x_start = nullptr, x_end = nullptr;
    cudaEvent_t in_done[3] = {}, run_done[3] = {}, out_done[3] = {};
    float2 *slot_s[3] = {}, *slot_y[3] = {};
    size_t slot_cap = 0;  // blocks per slot
    int slot_next = 0;    // next slot (the ring continues across calls)
    bool s_indep = false; // bf_filter_set_s_independent
    int variant = 5;      // bf_filter_set_variant (default: 12 warps per CTA, spectrum through L1)
    double tuned_us[7] = {};  // bf_filter_autotune: microseconds per launch of each variant (0: not timed)
    int64_t tuned_n_sig = 0;
    std::string device_name;
    int cc = 0;
};

static thread_local std::string g_create_err;

static bf_status ff_fail(bf_filter f, bf_status s, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    (f ? f->err : g_create_err) = buf;
    return s;
}

#define FF_CK(f, call)                                                                     \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess) {                                                           \
            cudaGetLastError();                                                            \
            return ff_fail(f, BF_ECUDA, "%s: %s", #call, cudaGetErrorString(e_));          \
        }                                                                                  \
    } while (0)

static bf_status ff_device(bf_filter f) {
    int cur = -1;
    FF_CK(f, cudaGetDevice(&cur));
    if (cur != f->device) FF_CK(f, cudaSetDevice(f->device));
    return BF_OK;
}

// Filter launches may start while the previous kernel on the stream finishes
// (see bf_filter_kernel); the spectrum launch releases its dependents only by
// completing, so a filter launch never reads a spectrum still being written.
// Hn = H / N (1/N is a power of two: exact)
__global__ void bf_scale_spectrum_kernel(const float2 *H, float2 *Hn) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const float2 h = H[i];
    Hn[i] = make_float2(h.x * (1.f / N), h.y * (1.f / N));
}

// The building blocks a filter can run (bf_filter_set_variant): the two-pass
// kernel with 11, 10 or 12 warps per CTA and the spectrum read through L1
// (which keeps them within the 168 registers a thread that 10 to 12 warps
// allow: read from shared memory, 10 and 11 warps spilled), or 8 or 6 warps
// per CTA with the spectrum in shared memory (bit-identical results), the
// three-pass kernel with four
// 128-thread teams per CTA, and the two-pass pair kernel with eight pairs of
// warps per CTA (variant 6).
constexpr int N_VARIANTS = 7;
static_assert(N_VARIANTS == sizeof(bf_filter_s::tuned_us) / sizeof(double), "one tuned time per variant");

template <bool FILTER, int WARPS, bool HG = false>
static cudaError_t launch_warp(const float2 *s, float2 *y, long long n_sig, const bf_filter f, cudaStream_t st,
                               bool s_indep) {
    const long long want = (n_sig + WARPS - 1) / WARPS;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)std::min<long long>(want, (long long)f->sm_count));
    cfg.blockDim = dim3(32 * WARPS);
    cfg.dynamicSmemBytes = wsmem_bytes(WARPS, HG);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = FILTER ? 1 : 0;  // the spectrum launch waits for everything before it
    return cudaLaunchKernelEx(&cfg, bf_filter_warp_kernel<FILTER, WARPS, HG>, s, y, n_sig, (const float2 *)f->tb,
                              (const float2 *)(FILTER ? f->H : nullptr), s_indep ? 1 : 0, (const float2 *)f->Hn);
}

template <int PAIRS>
static cudaError_t launch_pair(const float2 *s, float2 *y, long long n_sig, const bf_filter f, cudaStream_t st,
                               bool s_indep) {
    const long long want = (n_sig + PAIRS - 1) / PAIRS;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)std::min<long long>(want, (long long)f->sm_count));
    cfg.blockDim = dim3(64 * PAIRS);
    cfg.dynamicSmemBytes = psmem_bytes(PAIRS);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, bf_filter_pair_kernel<PAIRS>, s, y, n_sig, (const float2 *)f->tb,
                              (const float2 *)f->H, s_indep ? 1 : 0);
}

template <int PAIRS>
static cudaError_t configure_pair() {
    return cudaFuncSetAttribute(bf_filter_pair_kernel<PAIRS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                psmem_bytes(PAIRS));
}

template <bool FILTER, int WARPS, bool HG = false>
static cudaError_t configure_warp() {
    return cudaFuncSetAttribute(bf_filter_warp_kernel<FILTER, WARPS, HG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                wsmem_bytes(WARPS, HG));
}

// filter = false: y = FFT(s), always by the two-pass kernel, so the spectrum
// of the taps is the same whatever variant filters the blocks.
static cudaError_t launch_filter(bool filter, const float2 *s, float2 *y, long long n_sig, const bf_filter f,
                                 cudaStream_t st, bool s_indep = false, int variant = -1) {
    if (n_sig <= 0) return cudaSuccess;
    if (!filter) return launch_warp<false, 11>(s, y, n_sig, f, st, false);
    switch (variant < 0 ? f->variant : variant) {
        case 1: return launch_warp<true, 10, true>(s, y, n_sig, f, st, s_indep);
        case 2: return launch_warp<true, 8>(s, y, n_sig, f, st, s_indep);
        case 3: return launch_warp<true, 6>(s, y, n_sig, f, st, s_indep);
        case 5: return launch_warp<true, 12, true>(s, y, n_sig, f, st, s_indep);
        case 6: return launch_pair<8>(s, y, n_sig, f, st, s_indep);
        case 4: break;
        default: return launch_warp<true, 11, true>(s, y, n_sig, f, st, s_indep);
    }
    const long long want = (n_sig + TEAMS - 1) / TEAMS;
    const int grid = (int)std::min<long long>(want, (long long)f->sm_count * CTAS_PER_SM);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(THREADS);
    cfg.dynamicSmemBytes = SMEM_BYTES;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, bf_filter_kernel<true>, s, y, n_sig, (const float2 *)f->tw, (const float2 *)f->H,
                              s_indep ? 1 : 0);
}

extern "C" bf_status bf_filter_create(int n, bf_filter *out) {
    if (!out) return ff_fail(nullptr, BF_EINVAL, "out is NULL");
    *out = nullptr;
    if (n != N) return ff_fail(nullptr, BF_EINVAL, "n = %d: the filter is built for 2048-point transforms", n);
    int dev = 0;
    cudaDeviceProp prop;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
        cudaGetLastError();
        return ff_fail(nullptr, BF_ECUDA, "no usable CUDA device");
    }
    if (prop.major < 10) return ff_fail(nullptr, BF_ECUDA, "device sm_%d%d is not a Blackwell part", prop.major,
                                        prop.minor);
    bf_filter f = new bf_filter_s();
    f->device = dev;
    f->sm_count = prop.multiProcessorCount;
    f->device_name = prop.name;
    f->cc = prop.major * 10 + prop.minor;
    // per-pass twiddles e^{-2 pi i e / N}, from FP64 values rounded once to FP32
    std::vector<float2> tw(N, make_float2(0.f, 0.f));
    auto root = [](int e) {
        const double a = 2.0 * 3.14159265358979323846 * (double)(e % N) / (double)N;
        return make_float2((float)std::cos(a), (float)-std::sin(a));
    };
    for (int k = 0; k < 16; ++k) {
        tw[k] = root(8 * k);        // e^{-2 pi i k / 256}
        tw[16 + k] = root(32 * k);  // e^{-2 pi i 4 k / 256}
    }
    for (int j = 0; j < 256; ++j) tw[TW3 + j] = root(j);  // e^{-2 pi i j / 2048}
    std::vector<float2> tb(TB_SIZE, make_float2(0.f, 0.f));
    for (int a = 0; a < 64; ++a)
        for (int b = 0; b < 32; ++b) tb[a * TB_ROW + b] = root(a * b);  // e^{-2 pi i a b / 2048}
    bool ok = cudaMalloc((void **)&f->tw, N * sizeof(float2)) == cudaSuccess &&
              cudaMalloc((void **)&f->H, N * sizeof(float2)) == cudaSuccess &&
              cudaMalloc((void **)&f->hpad, N * sizeof(float2)) == cudaSuccess &&
              cudaMalloc((void **)&f->tb, TB_SIZE * sizeof(float2)) == cudaSuccess &&
              cudaMemcpy(f->tw, tw.data(), N * sizeof(float2), cudaMemcpyHostToDevice) == cudaSuccess &&
              cudaMemcpy(f->tb, tb.data(), TB_SIZE * sizeof(float2), cudaMemcpyHostToDevice) == cudaSuccess &&
              configure_warp<false, 11>() == cudaSuccess && configure_warp<true, 11, true>() == cudaSuccess &&
              configure_warp<true, 10, true>() == cudaSuccess && configure_warp<true, 8>() == cudaSuccess &&
              configure_warp<true, 6>() == cudaSuccess && configure_warp<true, 12, true>() == cudaSuccess &&
              configure_pair<8>() == cudaSuccess &&
              cudaMalloc((void **)&f->Hn, N * sizeof(float2)) == cudaSuccess &&
              cudaFuncSetAttribute(bf_filter_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   SMEM_BYTES) == cudaSuccess &&
              cudaStreamCreateWithFlags(&f->x_in, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&f->x_run, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&f->x_out, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&f->x_start, cudaEventDisableTiming) == cudaSuccess &&
              cudaEventCreateWithFlags(&f->x_end, cudaEventDisableTiming) == cudaSuccess;
    for (int i = 0; ok && i < 3; ++i)
        ok = cudaEventCreateWithFlags(&f->in_done[i], cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&f->run_done[i], cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&f->out_done[i], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        bf_filter_destroy(f);
        return ff_fail(nullptr, BF_ECUDA, "filter allocation or setup failed");
    }
    *out = f;
    return BF_OK;
}

extern "C" bf_status bf_filter_destroy(bf_filter f) {
    if (!f) return BF_OK;
    cudaSetDevice(f->device);
    cudaDeviceSynchronize();
    cudaGetLastError();
    for (void *p : {(void *)f->tw, (void *)f->H, (void *)f->hpad, (void *)f->tb, (void *)f->Hn})
        if (p) cudaFree(p);
    for (int i = 0; i < 3; ++i) {
        if (f->slot_s[i]) cudaFree(f->slot_s[i]);
        if (f->slot_y[i]) cudaFree(f->slot_y[i]);
        for (cudaEvent_t e : {f->in_done[i], f->run_done[i], f->out_done[i]})
            if (e) cudaEventDestroy(e);
    }
    for (cudaEvent_t e : {f->x_start, f->x_end})
        if (e) cudaEventDestroy(e);
    for (cudaStream_t s : {f->x_in, f->x_run, f->x_out})
        if (s) cudaStreamDestroy(s);
    cudaGetLastError();
    delete f;
    return BF_OK;
}

extern "C" const char *bf_filter_last_error(bf_filter f) { return f ? f->err.c_str() : g_create_err.c_str(); }

extern "C" int64_t bf_filter_launch_count(bf_filter f) { return f ? f->launches : 0; }

extern "C" bf_status bf_filter_set_taps(bf_filter f, const void *h_dev, int n_taps, void *stream) {
    if (!f) return ff_fail(nullptr, BF_EINVAL, "filter is NULL");
    if (!h_dev || n_taps < 1 || n_taps > N)
        return ff_fail(f, BF_EINVAL, "need 1 <= n_taps <= %d and a non-NULL h_dev (n_taps = %d)", N, n_taps);
    if ((uintptr_t)h_dev & 7u) return ff_fail(f, BF_EINVAL, "h_dev must be 8-byte aligned");
    bf_status s = ff_device(f);
    if (s != BF_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    FF_CK(f, cudaMemsetAsync(f->hpad, 0, N * sizeof(float2), st));
    FF_CK(f, cudaMemcpyAsync(f->hpad, h_dev, (size_t)n_taps * sizeof(float2), cudaMemcpyDeviceToDevice, st));
    FF_CK(f, launch_filter(false, f->hpad, f->H, 1, f, st));
    f->launches++;
    bf_scale_spectrum_kernel<<<N / 256, 256, 0, st>>>(f->H, f->Hn);
    FF_CK(f, cudaGetLastError());
    f->launches++;
    f->has_taps = true;
    return BF_OK;
}

extern "C" bf_status bf_filter_spectrum(bf_filter f, void *H_dev, void *stream) {
    if (!f) return ff_fail(nullptr, BF_EINVAL, "filter is NULL");
    if (!H_dev || ((uintptr_t)H_dev & 7u)) return ff_fail(f, BF_EINVAL, "H_dev must be non-NULL and 8-byte aligned");
    if (!f->has_taps) return ff_fail(f, BF_ENOTFOUND, "no filter sequence set");
    bf_status s = ff_device(f);
    if (s != BF_OK) return s;
    FF_CK(f, cudaMemcpyAsync(H_dev, f->H, N * sizeof(float2), cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
    return BF_OK;
}

static bf_status ff_check_apply(bf_filter f, const void *s, int64_t n_sig, const void *y, bool dev) {
    if (!f) return ff_fail(nullptr, BF_EINVAL, "filter is NULL");
    if (n_sig < 0) return ff_fail(f, BF_EINVAL, "negative n_sig");
    if (!f->has_taps) return ff_fail(f, BF_ENOTFOUND, "no filter sequence set");
    if (n_sig == 0) return BF_OK;
    if (!s || !y) return ff_fail(f, BF_EINVAL, "NULL buffer");
    if (dev && (((uintptr_t)s & 15u) || ((uintptr_t)y & 15u)))
        return ff_fail(f, BF_EINVAL, "s_dev and y_dev must be 16-byte aligned");
    if (s != y) {
        const uint8_t *a = (const uint8_t *)s, *b = (const uint8_t *)y;
        const size_t bytes = (size_t)n_sig * N * sizeof(float2);
        if (a < b + bytes && b < a + bytes) return ff_fail(f, BF_EINVAL, "s and y overlap without being equal");
    }
    return BF_OK;
}

extern "C" bf_status bf_filter_apply(bf_filter f, const void *s_dev, int64_t n_sig, void *y_dev, void *stream) {
    bf_status s = ff_check_apply(f, s_dev, n_sig, y_dev, true);
    if (s != BF_OK || n_sig == 0) return s;
    if ((s = ff_device(f)) != BF_OK) return s;
    FF_CK(f, launch_filter(true, (const float2 *)s_dev, (float2 *)y_dev, n_sig, f, (cudaStream_t)stream, f->s_indep));
    f->launches++;
    return BF_OK;
}

extern "C" bf_status bf_filter_set_s_independent(bf_filter f, int32_t independent) {
    if (!f) return ff_fail(nullptr, BF_EINVAL, "filter is NULL");
    if (independent != 0 && independent != 1) return ff_fail(f, BF_EINVAL, "independent must be 0 or 1");
    f->s_indep = independent != 0;
    return BF_OK;
}

// Chunks grow from 256 blocks (2 MiB in + 2 MiB out) to 2,048 blocks, so that
// the first copy-out starts early and later chunks amortise the calls. A
// slot's reuse waits for the kernel and the copy-out that last used it, in
// this call or an earlier one, so calls on different streams pipeline.
extern "C" bf_status bf_filter_apply_host(bf_filter f, const void *s_host, int64_t n_sig, void *y_host,
                                          void *stream) {
    bf_status s = ff_check_apply(f, s_host, n_sig, y_host, false);
    if (s != BF_OK || n_sig == 0) return s;
    if ((s = ff_device(f)) != BF_OK) return s;
    constexpr int64_t FIRST = 256, MAXC = 2048;
    const size_t need = (size_t)std::min<int64_t>(MAXC, n_sig);
    if (need > f->slot_cap) {
        FF_CK(f, cudaDeviceSynchronize());
        for (int i = 0; i < 3; ++i) {
            if (f->slot_s[i]) cudaFree(f->slot_s[i]);
            if (f->slot_y[i]) cudaFree(f->slot_y[i]);
            f->slot_s[i] = f->slot_y[i] = nullptr;
        }
        f->slot_cap = 0;
        for (int i = 0; i < 3; ++i) {
            FF_CK(f, cudaMalloc((void **)&f->slot_s[i], need * N * sizeof(float2)));
            FF_CK(f, cudaMalloc((void **)&f->slot_y[i], need * N * sizeof(float2)));
        }
        f->slot_cap = need;
    }
    cudaStream_t user = (cudaStream_t)stream;
    FF_CK(f, cudaEventRecord(f->x_start, user));
    FF_CK(f, cudaStreamWaitEvent(f->x_in, f->x_start, 0));
    FF_CK(f, cudaStreamWaitEvent(f->x_run, f->x_start, 0));
    FF_CK(f, cudaStreamWaitEvent(f->x_out, f->x_start, 0));
    const size_t blk = N * sizeof(float2);
    int64_t done = 0, chunk = FIRST;
    while (done < n_sig) {
        const int k = f->slot_next;
        f->slot_next = (f->slot_next + 1) % 3;
        const int64_t nb = std::min<int64_t>(std::min<int64_t>(chunk, (int64_t)f->slot_cap), n_sig - done);
        FF_CK(f, cudaStreamWaitEvent(f->x_in, f->run_done[k], 0));
        FF_CK(f, cudaMemcpyAsync(f->slot_s[k], (const uint8_t *)s_host + done * blk, nb * blk, cudaMemcpyHostToDevice,
                                 f->x_in));
        FF_CK(f, cudaEventRecord(f->in_done[k], f->x_in));
        FF_CK(f, cudaStreamWaitEvent(f->x_run, f->in_done[k], 0));
        FF_CK(f, cudaStreamWaitEvent(f->x_run, f->out_done[k], 0));
        FF_CK(f, launch_filter(true, f->slot_s[k], f->slot_y[k], nb, f, f->x_run));
        f->launches++;
        FF_CK(f, cudaEventRecord(f->run_done[k], f->x_run));
        FF_CK(f, cudaStreamWaitEvent(f->x_out, f->run_done[k], 0));
        FF_CK(f, cudaMemcpyAsync((uint8_t *)y_host + done * blk, f->slot_y[k], nb * blk, cudaMemcpyDeviceToHost,
                                 f->x_out));
        FF_CK(f, cudaEventRecord(f->out_done[k], f->x_out));
        done += nb;
        chunk = std::min<int64_t>(2 * chunk, MAXC);
    }
    FF_CK(f, cudaEventRecord(f->x_end, f->x_out));
    FF_CK(f, cudaStreamWaitEvent(user, f->x_end, 0));
    return BF_OK;
}

// ------------------------------------------------------------------ building blocks and their tuning

extern "C" bf_status bf_filter_set_variant(bf_filter f, int32_t variant) {
    if (!f) return ff_fail(nullptr, BF_EINVAL, "filter is NULL");
    if (variant < 0 || variant >= N_VARIANTS)
        return ff_fail(f, BF_EINVAL, "variant %d is outside [0, %d)", variant, N_VARIANTS);
    f->variant = variant;
    return BF_OK;
}

extern "C" int32_t bf_filter_get_variant(bf_filter f) { return f ? f->variant : -1; }

// Times every variant on n_sig synthetic blocks (scratch allocated and freed
// here) in the launch form the filter uses (s declared independent or not;
// the scratch input is never written during the timing, so independent
// launches are correct here too) and keeps the fastest.
extern "C" bf_status bf_filter_autotune(bf_filter f, int64_t n_sig, void *stream) {
    if (!f) return ff_fail(nullptr, BF_EINVAL, "filter is NULL");
    if (n_sig < 1 || n_sig > (1 << 20)) return ff_fail(f, BF_EINVAL, "n_sig = %lld is outside [1, 2^20]",
                                                       (long long)n_sig);
    if (!f->has_taps) return ff_fail(f, BF_ENOTFOUND, "no filter sequence set");
    bf_status st = ff_device(f);
    if (st != BF_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t bytes = (size_t)n_sig * N * sizeof(float2);
    float2 *a = nullptr, *b = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    auto cleanup = [&] {
        if (a) cudaFree(a);
        if (b) cudaFree(b);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        cudaGetLastError();
    };
    if (cudaMalloc((void **)&a, bytes) != cudaSuccess || cudaMalloc((void **)&b, bytes) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cleanup();
        return ff_fail(f, BF_ENOMEM, "autotune scratch (%zu bytes twice) could not be allocated", bytes);
    }
    double us[N_VARIANTS] = {};
    cudaError_t e = cudaMemsetAsync(a, 0x3C, bytes, s);  // finite values (about 0.0115 as FP32)
    constexpr int WARM = 3, REPS = 10, ROUNDS = 3;
    for (int v = 0; v < N_VARIANTS && e == cudaSuccess; ++v) {
        double best = 0.0;
        for (int r = 0; r < ROUNDS && e == cudaSuccess; ++r) {
            for (int i = 0; i < WARM && e == cudaSuccess; ++i) e = launch_filter(true, a, b, n_sig, f, s, f->s_indep, v);
            if (e == cudaSuccess) e = cudaEventRecord(e0, s);
            for (int i = 0; i < REPS && e == cudaSuccess; ++i) e = launch_filter(true, a, b, n_sig, f, s, f->s_indep, v);
            if (e == cudaSuccess) e = cudaEventRecord(e1, s);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            const double t = ms * 1e3 / REPS;
            if (e == cudaSuccess && (r == 0 || t < best)) best = t;
        }
        f->launches += ROUNDS * (WARM + REPS);
        us[v] = best;
    }
    cleanup();
    if (e != cudaSuccess) return ff_fail(f, BF_ECUDA, "filter autotune: %s", cudaGetErrorString(e));
    int pick = 0;
    for (int v = 1; v < N_VARIANTS; ++v)
        if (us[v] < us[pick]) pick = v;
    for (int v = 0; v < N_VARIANTS; ++v) f->tuned_us[v] = us[v];
    f->tuned_n_sig = n_sig;
    f->variant = pick;
    return BF_OK;
}

extern "C" bf_status bf_filter_tune_query(bf_filter f, int32_t variant, double *us_per_launch, int64_t *n_sig) {
    if (!f) return ff_fail(nullptr, BF_EINVAL, "filter is NULL");
    if (variant < 0 || variant >= N_VARIANTS) return ff_fail(f, BF_EINVAL, "variant %d is out of range", variant);
    if (us_per_launch) *us_per_launch = f->tuned_us[variant];
    if (n_sig) *n_sig = f->tuned_n_sig;
    return BF_OK;
}

extern "C" bf_status bf_filter_tune_save(bf_filter f, const char *path) {
    if (!f || !path) return ff_fail(f, BF_EINVAL, "NULL argument");
    FILE *fh = fopen(path, "w");
    if (!fh) return ff_fail(f, BF_EINVAL, "cannot open %s for writing", path);
    std::string name = f->device_name;
    for (char &ch : name)
        if (ch == '"' || ch == '\\' || (unsigned char)ch < 0x20) ch = '_';
    fprintf(fh, "{\n  \"format\": \"libbf-tune-2\",\n  \"kind\": \"filter\",\n");
    fprintf(fh, "  \"target\": {\"device\": \"%s\", \"cc\": %d, \"sm_count\": %d},\n", name.c_str(), f->cc,
            f->sm_count);
    fprintf(fh, "  \"n\": %d,\n  \"n_sig\": %lld,\n  \"variant\": %d,\n  \"us_per_launch\": [", N,
            (long long)f->tuned_n_sig, f->variant);
    for (int v = 0; v < N_VARIANTS; ++v) fprintf(fh, "%s%.4f", v ? ", " : "", f->tuned_us[v]);
    fprintf(fh, "]\n}\n");
    return fclose(fh) == 0 ? BF_OK : ff_fail(f, BF_EINVAL, "write to %s failed", path);
}

extern "C" bf_status bf_filter_tune_load(bf_filter f, const char *path) {
    if (!f || !path) return ff_fail(f, BF_EINVAL, "NULL argument");
    if (bf_tune_check_target(path, f->device_name.c_str(), f->cc, f->sm_count) != BF_OK)
        return ff_fail(f, BF_EINVAL, "%s", bf_last_error(nullptr));
    FILE *fh = fopen(path, "r");
    if (!fh) return ff_fail(f, BF_EINVAL, "cannot open %s", path);
    std::string txt;
    char buf[4096];
    size_t n;
    while ((n = fread(buf, 1, sizeof buf, fh)) > 0) txt.append(buf, n);
    fclose(fh);
    auto bad = [&](const char *why) { return ff_fail(f, BF_EINVAL, "%s: %s", path, why); };
    if (txt.find("\"kind\": \"filter\"") == std::string::npos) return bad("not a filter tune table");
    int nn = 0, variant = -1;
    long long ns = 0;
    size_t p = txt.find("\"n\":");
    if (p == std::string::npos || sscanf(txt.c_str() + p + 4, "%d", &nn) != 1 || nn != N) return bad("n");
    p = txt.find("\"n_sig\":");
    if (p == std::string::npos || sscanf(txt.c_str() + p + 8, "%lld", &ns) != 1 || ns < 0) return bad("n_sig");
    p = txt.find("\"variant\":");
    if (p == std::string::npos || sscanf(txt.c_str() + p + 10, "%d", &variant) != 1 || variant < 0 ||
        variant >= N_VARIANTS)
        return bad("variant");
    p = txt.find("\"us_per_launch\": [");
    if (p == std::string::npos) return bad("us_per_launch");
    double us[N_VARIANTS];
    const char *c = txt.c_str() + p + 18;
    for (int v = 0; v < N_VARIANTS; ++v) {
        char *end = nullptr;
        us[v] = strtod(c, &end);
        if (end == c || us[v] < 0) return bad("us_per_launch value");
        c = end + (*end == ',' ? 1 : 0);
    }
    f->variant = variant;
    f->tuned_n_sig = ns;
    for (int v = 0; v < N_VARIANTS; ++v) f->tuned_us[v] = us[v];
    return BF_OK;
}
