// bf_prep.h -- host-visible descriptors and launchers of the prep kernels.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace bfi {

struct PrecJob {       // one precoder to convert
    int64_t w_off;     // complex-element offset of its n_ant x f matrix in W
    int32_t f;
    int32_t slot;
};

struct QGroup {        // one group of S blocks to encode
    int64_t s_off;     // byte offset of the first complex64 block
    int64_t q_off;     // byte offset of the first held block
    int32_t f;
    int32_t nb;
    int32_t blk0;      // index of the first block in group order (scale index)
    int32_t pad;
};

cudaError_t launch_precoders(const float2 *W, const PrecJob *jobs, int n_jobs, uint8_t *w_simt,
                             uint8_t *w_bf16x2, uint8_t *w_fp16, uint8_t *w_tf32x2, float *w_scale,
                             cudaStream_t st);
cudaError_t launch_quantize(int prec, const uint8_t *S, const QGroup *groups, int n_groups, int max_nb,
                            uint8_t *Sq, float *scale_out, cudaStream_t st);
cudaError_t launch_selftest_wait(int *status, int *out, cudaStream_t st);
cudaError_t launch_errnorm(const float2 *R, const double2 *Rref, int64_t n_blocks, double *per_block,
                           double *total, int grid, cudaStream_t st);

struct KParams;
cudaError_t launch_simt(const KParams &p, int n_cta, cudaStream_t stream, bool three_products);
cudaError_t launch_tc(int prec, bool held, const KParams &p, int n_cta, cudaStream_t stream);
int simt_smem_bytes();
int simt_resident_ctas(bool g3m);
int tc_smem_bytes(int prec, bool held);
cudaError_t configure_simt();
cudaError_t configure_tc();

}  // namespace bfi
