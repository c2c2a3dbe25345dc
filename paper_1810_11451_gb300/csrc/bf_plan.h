// bf_plan.h -- the plan object behind the C ABI (host side only).
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <mutex>
#include <cstdint>
#include <string>
#include <vector>

#include "bf.h"
#include "bf_internal.h"

namespace bfi {

// Autotune table. Per precision and f bucket: the measured marginal cost of
// one block (ns, the slope of launch time over batch size) and the tile
// size (1 or 2 blocks) that measured faster. An untuned precision splits
// batches by bytes moved instead. Also the CTAs per SM of the CUDA-core kernel.
constexpr int TUNE_BUCKETS = 5;  // f in [0], [1,8], [9,16], [17,24], [25,36]
constexpr int TUNE_REP_F[TUNE_BUCKETS] = {0, 8, 16, 24, 36};
__host__ __device__ constexpr int f_bucket(int f) {
    return f <= 0 ? 0 : (f <= 8 ? 1 : (f <= 16 ? 2 : (f <= 24 ? 3 : 4)));
}

struct TuneTable {
    double ns_per_block[N_PREC][TUNE_BUCKETS];
    int tile_blocks[N_PREC][TUNE_BUCKETS];
    bool tuned[N_PREC] = {};
    int simt_ctas_per_sm[2] = {2, 2};  // plain, three-product form; the resident maximum at plan creation
    TuneTable() {
        for (int p = 0; p < N_PREC; ++p)
            for (int b = 0; b < TUNE_BUCKETS; ++b) {
                ns_per_block[p][b] = 0.0;
                tile_blocks[p][b] = 2;
            }
    }
    static int row(int prec) { return prec >= 0 && prec < N_PREC ? prec : 0; }
    int tile_blocks_for(int prec, int f) const { return tile_blocks[row(prec)][f_bucket(f)]; }
    // Scheduling cost of n blocks at f whose S and R take `bytes_per_block`.
    double cost(int prec, int f, int n, double bytes_per_block) const {
        return tuned[row(prec)] ? n * ns_per_block[row(prec)][f_bucket(f)] : n * bytes_per_block;
    }
};

struct WorkList {
    std::vector<Tile> tiles;      // capacity kept across calls; the first n_tiles are valid
    int n_tiles = 0;
    std::vector<int32_t> cta_begin;
    std::vector<double> cost;     // scheduling cost of one block, per group (scratch)
    std::vector<int64_t> bound;   // first block of each CTA's range (scratch)
};

// One work-list buffer of the ring: pinned host image, device copy, and the
// event recorded after the launch that reads it.
struct WorkBuf {
    uint8_t *d = nullptr;
    size_t cap = 0;
    uint8_t *h = nullptr;
    size_t hcap = 0;
    cudaEvent_t ev = nullptr;
    bool valid = false;
    size_t bytes = 0, tiles_bytes = 0;
};

// Staging of a precoder or quantisation job list: pinned host image, device
// copy, and the event recorded after the launch that reads it.
constexpr int PREP_RING = 8;
struct StageBuf {
    uint8_t *d = nullptr, *h = nullptr;
    size_t dcap = 0, hcap = 0;
    cudaEvent_t ev = nullptr;
};

}  // namespace bfi

// Host-buffer pipeline: staging slots and the S + R bytes of one chunk.
#ifndef BF_XFER_SLOTS
#define BF_XFER_SLOTS 3
#endif
#ifndef BF_HOST_CHUNK_BYTES
#define BF_HOST_CHUNK_BYTES (32 << 20)
#endif
#ifndef BF_HOST_CHUNK_FIRST
#define BF_HOST_CHUNK_FIRST (4 << 20)
#endif

struct bf_plan_s {
    int device = 0, sm_count = 0, n_ant = 64, f_max = 36, b = 60;
    int cc = 0;                 // compute capability, major * 10 + minor
    std::string device_name;    // cudaDeviceProp::name (the tune table's target)
    int simt_resident[2] = {2, 2};  // CTAs of the CUDA-core kernels (plain, three-product) that fit on one SM
    std::string err;
    std::mutex err_mu;  // err is written from the caller's and a serving engine's threads
    // precoder store (slots)
    int cap = 0;
    std::vector<int> f_slot;  // -1 = unset
    uint8_t *w_simt = nullptr, *w_bf16x2 = nullptr, *w_fp16 = nullptr, *w_tf32x2 = nullptr;
    float *w_scale = nullptr;
    int *d_status = nullptr;
    // work-list ring
    bfi::WorkBuf ring[64];  // one per call in flight; also caches repeated lists
    int ring_next = 0;
    bfi::WorkList scratch_wl;
    // prep staging: a ring, so that a call waits only for the launch that
    // last read the buffer it takes (precoder updates come in bursts)
    bfi::StageBuf prep[bfi::PREP_RING];
    int prep_next = 0;
    // buffers replaced by growth on latency-bound paths, freed with the plan
    std::vector<void *> retired_dev;
    std::vector<uint8_t *> retired_host;
    // accuracy report
    double *en_d = nullptr;
    uint8_t *en_h = nullptr;
    size_t en_cap = 0, en_hcap = 0;
    // graph capture
    cudaStream_t cap_stream = nullptr;
    // host-buffer pipeline: a copy-in, a compute and a copy-out stream over a
    // ring of BF_XFER_SLOTS device staging slots (S and R of one chunk each)
    cudaStream_t x_in = nullptr, x_run = nullptr, x_out = nullptr;
    cudaEvent_t x_start = nullptr, x_end = nullptr;
    cudaEvent_t x_in_done[BF_XFER_SLOTS] = {}, x_run_done[BF_XFER_SLOTS] = {}, x_out_done[BF_XFER_SLOTS] = {};
    uint8_t *x_s[BF_XFER_SLOTS] = {}, *x_r[BF_XFER_SLOTS] = {};
    size_t x_scap[BF_XFER_SLOTS] = {}, x_rcap[BF_XFER_SLOTS] = {};
    int x_next = 0;  // next staging slot (the ring continues across calls)
    int64_t host_chunk_first = BF_HOST_CHUNK_FIRST, host_chunk_bytes = BF_HOST_CHUNK_BYTES;
    // tuning and counters
    bfi::TuneTable tune;
    int64_t launches = 0;
    std::atomic<int> servers{0};  // serving engines attached to this plan
};

bf_status bf_fail(bf_plan plan, bf_status s, const char *fmt, ...);
bf_status plan_ensure_device(bf_plan plan);
void build_worklist(const int *f_slot, const bfi::TuneTable &tune, const bf_group *groups, int32_t n_groups,
                    bf_precision prec, bool held, int max_cta, int64_t r_block_stride, bfi::WorkList &wl);
// `layout` nullptr = packed block-major complex64 R; otherwise already validated.
bf_status enqueue_apply(bf_plan plan, const void *S, const float *scale, const bf_group *groups, int32_t n_groups,
                        bf_precision prec, void *R, cudaStream_t st, int max_cta, const bf_rlayout *layout = nullptr);
int max_cta_for(bf_plan plan, bf_precision prec);
cudaError_t launch_kernel(bf_precision prec, bool held, const bfi::KParams &p, int n_cta, cudaStream_t st);
