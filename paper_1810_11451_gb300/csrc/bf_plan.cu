// bf_plan.cu -- host side of libbf: plans, the precoder store, the work-list
// scheduler, launches, prepared (graph-captured) batches, the host-buffer
// pipeline and the accuracy report. The C ABI is declared in include/bf.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "bf_internal.h"
#include "bf_plan.h"
#include "bf_prep.h"

using namespace bfi;

static thread_local std::string g_err;  // errors with no plan (creation)

bf_status bf_fail(bf_plan plan, bf_status s, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (plan) {
        std::lock_guard<std::mutex> g(plan->err_mu);  // a serving engine fails from two threads
        plan->err = buf;
    } else {
        g_err = buf;
    }
    return s;
}

#define BF_CK(plan, call)                                                                    \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess)                                                               \
            return bf_fail((plan), BF_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

// ------------------------------------------------------------------ small helpers
static bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

bf_status plan_ensure_device(bf_plan plan) {
    int cur = -1;
    BF_CK(plan, cudaGetDevice(&cur));
    if (cur != plan->device) BF_CK(plan, cudaSetDevice(plan->device));
    return BF_OK;
}

// Grow a device buffer to at least `need` bytes (doubling). The old buffer is
// freed after a device synchronisation, or with `retire` kept until the plan
// is destroyed, so that a caller on a latency-bound path never synchronises
// the device (its last reader must have finished).
template <typename T>
static bf_status grow_dev(bf_plan plan, T **p, size_t *cap, size_t need, bool retire = false) {
    if (need <= *cap) return BF_OK;
    size_t n = std::max(need, *cap * 2);
    if (*p) {
        if (retire) {
            plan->retired_dev.push_back(*p);
        } else {
            BF_CK(plan, cudaDeviceSynchronize());
            BF_CK(plan, cudaFree(*p));
        }
        *p = nullptr;
        *cap = 0;
    }
    if (cudaMalloc((void **)p, n) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return bf_fail(plan, BF_ENOMEM, "cudaMalloc of %zu bytes failed", n);
    }
    *cap = n;
    return BF_OK;
}

// The same for pinned host memory.
static bf_status grow_pinned(bf_plan plan, uint8_t **p, size_t *cap, size_t need, bool retire = false) {
    if (need <= *cap) return BF_OK;
    size_t n = std::max(need, *cap * 2);
    if (*p) {
        if (retire) plan->retired_host.push_back(*p);
        else BF_CK(plan, cudaFreeHost(*p));
        *p = nullptr;
        *cap = 0;
    }
    if (cudaMallocHost((void **)p, n) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return bf_fail(plan, BF_ENOMEM, "cudaMallocHost of %zu bytes failed", n);
    }
    *cap = n;
    return BF_OK;
}

// ------------------------------------------------------------------ C ABI: plan
extern "C" const char *bf_status_string(bf_status s) {
    switch (s) {
        case BF_OK: return "BF_OK";
        case BF_EINVAL: return "BF_EINVAL";
        case BF_ENOMEM: return "BF_ENOMEM";
        case BF_EBUDGET: return "BF_EBUDGET";
        case BF_ECUDA: return "BF_ECUDA";
        case BF_ETIMEOUT: return "BF_ETIMEOUT";
        case BF_EAGAIN: return "BF_EAGAIN";
        case BF_EBUSY: return "BF_EBUSY";
        case BF_ENOTREADY: return "BF_ENOTREADY";
        case BF_ENOTFOUND: return "BF_ENOTFOUND";
    }
    return "BF_UNKNOWN";
}

extern "C" const char *bf_last_error(bf_plan plan) {
    if (!plan) return g_err.c_str();
    static thread_local std::string copy;  // stays valid in this thread while others fail
    std::lock_guard<std::mutex> g(plan->err_mu);
    copy = plan->err;
    return copy.c_str();
}

extern "C" bf_status bf_plan_create(int n_ant, int f_max, int b, bf_plan *out) {
    if (!out) return bf_fail(nullptr, BF_EINVAL, "out is NULL");
    *out = nullptr;
    if (n_ant != N_ANT) return bf_fail(nullptr, BF_EINVAL, "n_ant must be %d, got %d", N_ANT, n_ant);
    if (b != B_RE) return bf_fail(nullptr, BF_EINVAL, "b must be %d, got %d", B_RE, b);
    if (f_max < 0 || f_max > F_LIMIT)
        return bf_fail(nullptr, BF_EINVAL, "f_max must be in [0, %d], got %d", F_LIMIT, f_max);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return bf_fail(nullptr, BF_ECUDA, "no CUDA device: %s", cudaGetErrorString(e));
    cudaDeviceProp prop;
    e = cudaGetDeviceProperties(&prop, dev);
    if (e != cudaSuccess) return bf_fail(nullptr, BF_ECUDA, "cudaGetDeviceProperties: %s", cudaGetErrorString(e));
    if (prop.major != 10 || prop.minor != 3)
        return bf_fail(nullptr, BF_ECUDA, "libbf is built for sm_103a; device %d is sm_%d%d", dev, prop.major,
                       prop.minor);
    static bool configured = false;
    if (!configured) {
        if ((e = configure_simt()) != cudaSuccess || (e = configure_tc()) != cudaSuccess)
            return bf_fail(nullptr, BF_ECUDA, "kernel configuration: %s", cudaGetErrorString(e));
        configured = true;
    }
    bf_plan p = new bf_plan_s();
    p->device = dev;
    p->sm_count = prop.multiProcessorCount;
    p->cc = prop.major * 10 + prop.minor;
    p->device_name = prop.name;
    p->n_ant = n_ant;
    p->f_max = f_max;
    p->b = b;
    for (int g = 0; g < 2; ++g) p->tune.simt_ctas_per_sm[g] = p->simt_resident[g] = simt_resident_ctas(g == 1);
    if (cudaMalloc((void **)&p->d_status, 64) != cudaSuccess || cudaMemset(p->d_status, 0, 64) != cudaSuccess) {
        cudaGetLastError();
        delete p;
        return bf_fail(nullptr, BF_ENOMEM, "status word allocation failed");
    }
    for (auto &w : p->ring) {
        if (cudaEventCreateWithFlags(&w.ev, cudaEventDisableTiming) != cudaSuccess) {
            bf_plan_destroy(p);
            return bf_fail(nullptr, BF_ECUDA, "cudaEventCreate failed");
        }
    }
    bool ok = true;
    for (auto &b : p->prep) ok = ok && cudaEventCreateWithFlags(&b.ev, cudaEventDisableTiming) == cudaSuccess;
    ok = ok &&
              cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&p->x_in, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&p->x_run, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&p->x_out, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&p->x_start, cudaEventDisableTiming) == cudaSuccess &&
              cudaEventCreateWithFlags(&p->x_end, cudaEventDisableTiming) == cudaSuccess;
    for (int i = 0; ok && i < BF_XFER_SLOTS; ++i)
        ok = cudaEventCreateWithFlags(&p->x_in_done[i], cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&p->x_run_done[i], cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&p->x_out_done[i], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        bf_plan_destroy(p);
        return bf_fail(nullptr, BF_ECUDA, "stream/event creation failed");
    }
    *out = p;
    return BF_OK;
}

extern "C" bf_status bf_plan_destroy(bf_plan plan) {
    if (!plan) return BF_OK;
    if (plan->servers.load() > 0)
        return bf_fail(plan, BF_EBUSY, "%d serving engine(s) still use this plan", plan->servers.load());
    cudaSetDevice(plan->device);
    cudaDeviceSynchronize();
    cudaGetLastError();
    for (auto &w : plan->ring) {
        if (w.d) cudaFree(w.d);
        if (w.h) cudaFreeHost(w.h);
        if (w.ev) cudaEventDestroy(w.ev);
    }
    void *dev_ptrs[] = {plan->w_simt, plan->w_bf16x2, plan->w_fp16, plan->w_tf32x2, plan->w_scale,
                        plan->d_status, plan->en_d};
    for (void *q : dev_ptrs)
        if (q) cudaFree(q);
    for (int i = 0; i < BF_XFER_SLOTS; ++i) {
        if (plan->x_s[i]) cudaFree(plan->x_s[i]);
        if (plan->x_r[i]) cudaFree(plan->x_r[i]);
        for (cudaEvent_t e : {plan->x_in_done[i], plan->x_run_done[i], plan->x_out_done[i]})
            if (e) cudaEventDestroy(e);
    }
    for (auto &b : plan->prep) {
        if (b.d) cudaFree(b.d);
        if (b.h) cudaFreeHost(b.h);
        if (b.ev) cudaEventDestroy(b.ev);
    }
    for (void *q : plan->retired_dev) cudaFree(q);
    for (uint8_t *q : plan->retired_host) cudaFreeHost(q);
    if (plan->en_h) cudaFreeHost(plan->en_h);
    if (plan->x_start) cudaEventDestroy(plan->x_start);
    if (plan->x_end) cudaEventDestroy(plan->x_end);
    for (cudaStream_t st : {plan->cap_stream, plan->x_in, plan->x_run, plan->x_out})
        if (st) cudaStreamDestroy(st);
    cudaGetLastError();
    delete plan;
    return BF_OK;
}

extern "C" bf_status bf_device_status(bf_plan plan) {
    if (!plan) return bf_fail(nullptr, BF_EINVAL, "plan is NULL");
    bf_status s = plan_ensure_device(plan);
    if (s != BF_OK) return s;
    BF_CK(plan, cudaDeviceSynchronize());
    int v = 0;
    BF_CK(plan, cudaMemcpy(&v, plan->d_status, sizeof v, cudaMemcpyDeviceToHost));
    if (v) {
        BF_CK(plan, cudaMemset(plan->d_status, 0, sizeof v));
        return bf_fail(plan, BF_ETIMEOUT, "a kernel gave up on a bounded wait (status 0x%x)", v);
    }
    return BF_OK;
}

extern "C" bf_status bf_selftest_wait_timeout(bf_plan plan, int32_t *out_host) {
    if (!plan || !out_host) return bf_fail(plan, BF_EINVAL, "NULL argument");
    bf_status s = plan_ensure_device(plan);
    if (s != BF_OK) return s;
    BF_CK(plan, cudaDeviceSynchronize());
    // ints 4..7 of the 64-byte status block receive the four results
    int *out_dev = plan->d_status + 4;
    BF_CK(plan, cudaMemset(out_dev, 0, 4 * sizeof(int)));
    BF_CK(plan, launch_selftest_wait(plan->d_status, out_dev, nullptr));
    BF_CK(plan, cudaDeviceSynchronize());
    int v[4];
    BF_CK(plan, cudaMemcpy(v, out_dev, sizeof v, cudaMemcpyDeviceToHost));
    for (int i = 0; i < 4; ++i) out_host[i] = v[i];
    return BF_OK;
}

// ------------------------------------------------------------------ precoders
// The next staging buffer of the ring, with room for `bytes`; waits only if
// the launch that last read it has not run yet.
static bf_status prep_stage(bf_plan plan, size_t bytes, StageBuf **out) {
    StageBuf &b = plan->prep[plan->prep_next];
    plan->prep_next = (plan->prep_next + 1) % PREP_RING;
    BF_CK(plan, cudaEventSynchronize(b.ev));
    bf_status s;
    if ((s = grow_pinned(plan, &b.h, &b.hcap, bytes, true)) != BF_OK) return s;
    if ((s = grow_dev(plan, &b.d, &b.dcap, bytes, true)) != BF_OK) return s;
    *out = &b;
    return BF_OK;
}

static bf_status ensure_slots(bf_plan plan, int need) {
    if (need <= plan->cap) return BF_OK;
    int ncap = std::max(need, std::max(64, plan->cap * 2));
    uint8_t *ns = nullptr, *nb = nullptr, *nf = nullptr, *nt = nullptr;
    float *nsc = nullptr;
    const size_t bs = (size_t)ncap * W_SIMT_STRIDE, bb = (size_t)ncap * W_BF16X2_STRIDE,
                 bf = (size_t)ncap * W_FP16_STRIDE, bt = (size_t)ncap * W_TF32X2_STRIDE,
                 bsc = (size_t)ncap * sizeof(float);
    if (cudaMalloc((void **)&ns, bs) != cudaSuccess || cudaMalloc((void **)&nb, bb) != cudaSuccess ||
        cudaMalloc((void **)&nf, bf) != cudaSuccess || cudaMalloc((void **)&nt, bt) != cudaSuccess ||
        cudaMalloc((void **)&nsc, bsc) != cudaSuccess) {
        cudaGetLastError();
        if (ns) cudaFree(ns);
        if (nb) cudaFree(nb);
        if (nf) cudaFree(nf);
        if (nt) cudaFree(nt);
        if (nsc) cudaFree(nsc);
        return bf_fail(plan, BF_ENOMEM, "precoder store growth to %d slots failed", ncap);
    }
    BF_CK(plan, cudaDeviceSynchronize());
    if (plan->cap) {
        BF_CK(plan, cudaMemcpy(ns, plan->w_simt, (size_t)plan->cap * W_SIMT_STRIDE, cudaMemcpyDeviceToDevice));
        BF_CK(plan, cudaMemcpy(nb, plan->w_bf16x2, (size_t)plan->cap * W_BF16X2_STRIDE, cudaMemcpyDeviceToDevice));
        BF_CK(plan, cudaMemcpy(nf, plan->w_fp16, (size_t)plan->cap * W_FP16_STRIDE, cudaMemcpyDeviceToDevice));
        BF_CK(plan, cudaMemcpy(nt, plan->w_tf32x2, (size_t)plan->cap * W_TF32X2_STRIDE, cudaMemcpyDeviceToDevice));
        BF_CK(plan, cudaMemcpy(nsc, plan->w_scale, (size_t)plan->cap * sizeof(float), cudaMemcpyDeviceToDevice));
        cudaFree(plan->w_simt);
        cudaFree(plan->w_bf16x2);
        cudaFree(plan->w_fp16);
        cudaFree(plan->w_tf32x2);
        cudaFree(plan->w_scale);
    }
    plan->w_simt = ns;
    plan->w_bf16x2 = nb;
    plan->w_fp16 = nf;
    plan->w_tf32x2 = nt;
    plan->w_scale = nsc;
    plan->f_slot.resize(ncap, -1);
    plan->cap = ncap;
    return BF_OK;
}

extern "C" bf_status bf_get_precoder_image(bf_plan plan, int32_t slot, bf_image kind, void *host_out,
                                         int64_t capacity, int64_t *bytes_out) {
    if (!plan || !bytes_out) return bf_fail(plan, BF_EINVAL, "NULL argument");
    if (slot < 0 || slot >= plan->cap || plan->f_slot[slot] < 0)
        return bf_fail(plan, BF_ENOTFOUND, "precoder slot %d is not set", slot);
    const int f = plan->f_slot[slot];
    const uint8_t *src = nullptr;
    int64_t bytes = 0;
    switch (kind) {
        case BF_IMG_FP32:
            src = plan->w_simt + (int64_t)slot * W_SIMT_STRIDE;
            bytes = simt_img_bytes(f, 3);
            break;
        case BF_IMG_BF16X2:
            src = plan->w_bf16x2 + (int64_t)slot * W_BF16X2_STRIDE;
            bytes = 2 * (int64_t)tc_img_bytes(kpad_of(f));
            break;
        case BF_IMG_FP16:
            src = plan->w_fp16 + (int64_t)slot * W_FP16_STRIDE;
            bytes = tc_img_bytes(kpad_of(f));
            break;
        case BF_IMG_TF32X2:
            src = plan->w_tf32x2 + (int64_t)slot * W_TF32X2_STRIDE;
            bytes = 2 * (int64_t)tf32_img_bytes(kpad32_of(f));
            break;
        case BF_IMG_SCALE:
            src = reinterpret_cast<const uint8_t *>(plan->w_scale + slot);
            bytes = sizeof(float);
            break;
        default:
            return bf_fail(plan, BF_EINVAL, "unknown image kind %d", (int)kind);
    }
    *bytes_out = bytes;
    if (!host_out) return BF_OK;
    if (capacity < bytes) return bf_fail(plan, BF_EINVAL, "capacity %lld < %lld bytes", (long long)capacity,
                                         (long long)bytes);
    bf_status s = plan_ensure_device(plan);
    if (s != BF_OK) return s;
    BF_CK(plan, cudaDeviceSynchronize());
    BF_CK(plan, cudaMemcpy(host_out, src, (size_t)bytes, cudaMemcpyDeviceToHost));
    return BF_OK;
}

extern "C" bf_status bf_set_host_chunks(bf_plan plan, int64_t first_bytes, int64_t max_bytes) {
    if (!plan) return bf_fail(nullptr, BF_EINVAL, "plan is NULL");
    if (first_bytes < (1 << 16) || max_bytes < first_bytes || max_bytes > ((int64_t)1 << 34))
        return bf_fail(plan, BF_EINVAL, "chunk sizes must satisfy 64 KiB <= first <= max <= 16 GiB");
    plan->host_chunk_first = first_bytes;
    plan->host_chunk_bytes = max_bytes;
    return BF_OK;
}

extern "C" bf_status bf_reserve_worklists(bf_plan plan, int64_t max_blocks) {
    if (!plan) return bf_fail(nullptr, BF_EINVAL, "plan is NULL");
    if (max_blocks < 0 || max_blocks > (int64_t)1 << 30) return bf_fail(plan, BF_EINVAL, "max_blocks out of range");
    bf_status s = plan_ensure_device(plan);
    if (s != BF_OK) return s;
    // at most one tile per block, and one range start per CTA of any form
    const size_t bytes = (size_t)max_blocks * sizeof(Tile) + (size_t)(plan->sm_count * 16 + 1) * sizeof(int32_t);
    for (auto &w : plan->ring) {
        if (bytes <= w.hcap && bytes <= w.cap) continue;
        BF_CK(plan, cudaEventSynchronize(w.ev));
        w.valid = false;  // the new buffers do not hold the cached list
        if ((s = grow_pinned(plan, &w.h, &w.hcap, bytes, true)) != BF_OK) return s;
        if ((s = grow_dev(plan, &w.d, &w.cap, bytes, true)) != BF_OK) return s;
    }
    return BF_OK;
}

extern "C" bf_status bf_reserve_precoders(bf_plan plan, int32_t n_slots) {
    if (!plan) return bf_fail(nullptr, BF_EINVAL, "plan is NULL");
    if (n_slots < 0 || n_slots > (1 << 24)) return bf_fail(plan, BF_EINVAL, "n_slots out of range");
    bf_status s = plan_ensure_device(plan);
    if (s != BF_OK) return s;
    return ensure_slots(plan, n_slots);
}

extern "C" bf_status bf_set_precoders(bf_plan plan, const void *W_dev, const int32_t *f_host, int32_t n_prec,
                                      int32_t first_id, void *stream) {
    if (!plan) return bf_fail(nullptr, BF_EINVAL, "plan is NULL");
    if (n_prec < 0 || first_id < 0) return bf_fail(plan, BF_EINVAL, "negative n_prec or first_id");
    if (n_prec == 0) return BF_OK;
    if (!W_dev || !f_host) return bf_fail(plan, BF_EINVAL, "W_dev or f_host is NULL");
    if (((uintptr_t)W_dev & 7u) != 0) return bf_fail(plan, BF_EINVAL, "W_dev must be 8-byte aligned");
    if ((int64_t)first_id + n_prec > (1 << 24)) return bf_fail(plan, BF_EINVAL, "slot id too large");
    for (int i = 0; i < n_prec; ++i)
        if (f_host[i] < 0 || f_host[i] > plan->f_max)
            return bf_fail(plan, BF_EINVAL, "precoder %d: f = %d outside [0, f_max = %d]", i, f_host[i],
                           plan->f_max);
    bf_status s = plan_ensure_device(plan);
    if (s != BF_OK) return s;
    if ((s = ensure_slots(plan, first_id + n_prec)) != BF_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t bytes = (size_t)n_prec * sizeof(PrecJob);
    StageBuf *sb = nullptr;
    if ((s = prep_stage(plan, bytes, &sb)) != BF_OK) return s;
    PrecJob *jobs = reinterpret_cast<PrecJob *>(sb->h);
    int64_t off = 0;
    for (int i = 0; i < n_prec; ++i) {
        jobs[i].w_off = off;
        jobs[i].f = f_host[i];
        jobs[i].slot = first_id + i;
        off += (int64_t)N_ANT * f_host[i];
    }
    BF_CK(plan, cudaMemcpyAsync(sb->d, sb->h, bytes, cudaMemcpyHostToDevice, st));
    BF_CK(plan, launch_precoders(reinterpret_cast<const float2 *>(W_dev), reinterpret_cast<PrecJob *>(sb->d),
                                 n_prec, plan->w_simt, plan->w_bf16x2, plan->w_fp16, plan->w_tf32x2,
                                 plan->w_scale, st));
    BF_CK(plan, cudaEventRecord(sb->ev, st));
    for (int i = 0; i < n_prec; ++i) plan->f_slot[first_id + i] = f_host[i];
    return BF_OK;
}

// ------------------------------------------------------------------ held symbols
extern "C" int64_t bf_held_block_bytes(int f, bf_precision prec) {
    if (f < 0 || f > F_LIMIT) return 0;
    if (prec == BF_BF16 || prec == BF_FP16) return held_block_bytes(f, 1);
    if (prec == BF_BF16X3) return held_block_bytes(f, 2);
    return 0;
}

static bf_status check_group_slots(bf_plan plan, const bf_group *groups, int32_t n_groups) {
    for (int g = 0; g < n_groups; ++g) {
        const bf_group &gr = groups[g];
        if (gr.n_blocks < 0) return bf_fail(plan, BF_EINVAL, "group %d: negative n_blocks", g);
        if (gr.prec_id < 0 || gr.prec_id >= plan->cap || plan->f_slot[gr.prec_id] < 0)
            return bf_fail(plan, BF_ENOTFOUND, "group %d: precoder slot %d is not set", g, gr.prec_id);
        if (gr.s_off < 0 || gr.r_off < 0 || (gr.s_off & 15) || (gr.r_off & 15))
            return bf_fail(plan, BF_EINVAL, "group %d: offsets must be non-negative multiples of 16", g);
    }
    return BF_OK;
}

extern "C" bf_status bf_quantize_symbols(bf_plan plan, const void *S_dev, const bf_group *groups, int32_t n_groups,
                                         bf_precision prec, void *Sq_dev, const int64_t *q_off_host,
                                         float *scale_dev, void *stream) {
    if (!plan) return bf_fail(nullptr, BF_EINVAL, "plan is NULL");
    if (n_groups < 0) return bf_fail(plan, BF_EINVAL, "negative n_groups");
    if (prec != BF_BF16 && prec != BF_FP16 && prec != BF_BF16X3)
        return bf_fail(plan, BF_EINVAL, "held S exists for BF_BF16, BF_FP16 and BF_BF16X3 only");
    if (n_groups == 0) return BF_OK;
    if (!groups || !q_off_host || !S_dev || !Sq_dev || !scale_dev)
        return bf_fail(plan, BF_EINVAL, "NULL argument");
    if (!aligned16(S_dev) || !aligned16(Sq_dev) || ((uintptr_t)scale_dev & 3u))
        return bf_fail(plan, BF_EINVAL, "S_dev and Sq_dev must be 16-byte aligned");
    bf_status s = check_group_slots(plan, groups, n_groups);
    if (s != BF_OK) return s;
    for (int g = 0; g < n_groups; ++g)
        if (q_off_host[g] < 0 || (q_off_host[g] & 15))
            return bf_fail(plan, BF_EINVAL, "group %d: q_off must be a non-negative multiple of 16", g);
    if ((s = plan_ensure_device(plan)) != BF_OK) return s;
    const size_t bytes = (size_t)n_groups * sizeof(QGroup);
    StageBuf *sb = nullptr;
    if ((s = prep_stage(plan, bytes, &sb)) != BF_OK) return s;
    QGroup *q = reinterpret_cast<QGroup *>(sb->h);
    int blk = 0, max_nb = 0;
    for (int g = 0; g < n_groups; ++g) {
        q[g].s_off = groups[g].s_off;
        q[g].q_off = q_off_host[g];
        q[g].f = plan->f_slot[groups[g].prec_id];
        q[g].nb = groups[g].n_blocks;
        q[g].blk0 = blk;
        q[g].pad = 0;
        blk += groups[g].n_blocks;
        max_nb = std::max(max_nb, (int)groups[g].n_blocks);
    }
    cudaStream_t st = (cudaStream_t)stream;
    BF_CK(plan, cudaMemcpyAsync(sb->d, sb->h, bytes, cudaMemcpyHostToDevice, st));
    BF_CK(plan, launch_quantize(prec, (const uint8_t *)S_dev, reinterpret_cast<QGroup *>(sb->d), n_groups,
                                max_nb, (uint8_t *)Sq_dev, scale_dev, st));
    BF_CK(plan, cudaEventRecord(sb->ev, st));
    return BF_OK;
}

// ------------------------------------------------------------------ work lists
// The blocks of the batch, in group order, are split into n_cta contiguous
// ranges of about equal cost (measured ns per block once tuned, bytes moved
// before), at block granularity: CTA loads differ by at most about one block.
// Within a range, each group's run of blocks becomes tiles of up to
// tile_blocks consecutive blocks (the size per f bucket comes from the
// autotune table), so each CTA loads a precoder once per run and streams its
// S blocks.
void build_worklist(const int *f_slot, const TuneTable &tune, const bf_group *groups, int32_t n_groups,
                    bf_precision prec, bool held, int max_cta, int64_t r_block_stride, WorkList &wl) {
    // per-group block cost, and the total (the buffers persist across calls in
    // the plan, so steady-state scheduling allocates nothing)
    wl.cost.resize(n_groups);
    double *cost = wl.cost.data();
    double total = 0;
    int64_t n_blocks = 0;
    for (int g = 0; g < n_groups; ++g) {
        const int f = f_slot[groups[g].prec_id];
        const int64_t sb = held ? held_block_bytes(f, prec == BF_BF16X3 ? 2 : 1) : (int64_t)f * S_BYTES_PER_F;
        cost[g] = tune.cost(prec, f, 1, (double)(sb + R_BLOCK_BYTES));
        total += cost[g] * groups[g].n_blocks;
        n_blocks += groups[g].n_blocks;
    }
    wl.n_tiles = 0;
    if (n_blocks == 0) {  // nothing to launch: one empty range
        wl.cta_begin.assign(2, 0);
        return;
    }
    const int n_cta = (int)std::max<int64_t>(1, std::min<int64_t>(max_cta, n_blocks));
    // Midpoint rule: block k goes to CTA floor((cum_k + cost_k / 2) * n_cta /
    // total), so CTA c starts at the first block whose midpoint reaches
    // c * total / n_cta. One walk over the groups finds every start; then the
    // starts are made strictly increasing and leave every CTA a block.
    std::vector<int64_t> &bound = wl.bound;
    bound.assign(n_cta + 1, 0);
    bound[n_cta] = n_blocks;
    {
        int g = 0;
        double c0 = 0;  // cost before group g
        int64_t k0 = 0; // blocks before group g
        for (int c = 1; c < n_cta; ++c) {
            const double target = total * c / n_cta;
            while (g < n_groups && c0 + cost[g] * (groups[g].n_blocks - 0.5) < target) {
                c0 += cost[g] * groups[g].n_blocks;
                k0 += groups[g].n_blocks;
                ++g;
            }
            int64_t b = 0;
            if (g < n_groups && cost[g] > 0) {
                b = (int64_t)std::ceil((target - c0) / cost[g] - 0.5);
                b = std::min<int64_t>(std::max<int64_t>(b, 0), groups[g].n_blocks);
            }
            bound[c] = k0 + b;
        }
        for (int c = 1; c < n_cta; ++c) bound[c] = std::max(bound[c], bound[c - 1] + 1);
        for (int c = n_cta - 1; c >= 1; --c) bound[c] = std::min(bound[c], bound[c + 1] - 1);
    }
    // tiles: each group's blocks, cut at the range starts, in runs of up to
    // tile_blocks (at most one tile per block, so the arrays are sized once)
    if (wl.tiles.size() < (size_t)n_blocks) wl.tiles.resize((size_t)n_blocks);
    wl.cta_begin.resize((size_t)n_cta + 1);
    Tile *tiles = wl.tiles.data();
    int32_t *cta_begin = wl.cta_begin.data();
    const int64_t *bnd = bound.data();
    int n_tiles = 0;
    cta_begin[0] = 0;
    int cur = 0;
    int64_t k = 0;
    int blk = 0;
    // precoder-run flags within each CTA's range, counting tiles with f > 0
    // only, set as the tiles are made: the first tile of a run of one precoder
    // and the last one (closed when another precoder starts or the range ends)
    int prev = -1, last_idx = -1;
    auto close_range = [&] {
        if (last_idx >= 0) tiles[last_idx].flags |= TF_LAST_OF_W;
        prev = last_idx = -1;
    };
    for (int g = 0; g < n_groups; ++g) {
        const bf_group &gr = groups[g];
        const int f = f_slot[gr.prec_id];
        const int64_t sb = held ? held_block_bytes(f, prec == BF_BF16X3 ? 2 : 1) : (int64_t)f * S_BYTES_PER_F;
        const int tile_blocks = tune.tile_blocks_for(prec, f);
        int pos = 0;
        while (pos < gr.n_blocks) {
            while (cur + 1 < n_cta && bnd[cur + 1] <= k + pos) {  // a range starts here
                close_range();
                cta_begin[++cur] = n_tiles;
            }
            const int stop = cur + 1 < n_cta ? (int)std::min<int64_t>(gr.n_blocks, bnd[cur + 1] - k) : gr.n_blocks;
            const int32_t first_flag = (f > 0 && stop > pos && gr.prec_id != prev) ? TF_FIRST_OF_W : 0;
            if (f > 0 && stop > pos) {
                if (first_flag && last_idx >= 0) tiles[last_idx].flags |= TF_LAST_OF_W;
                prev = gr.prec_id;
            }
            int64_t s_off = gr.s_off + (int64_t)pos * sb, r_off = gr.r_off + (int64_t)pos * r_block_stride;
            const int64_t s_step = (int64_t)tile_blocks * sb, r_step = (int64_t)tile_blocks * r_block_stride;
            Tile *t = tiles + n_tiles;
            for (int b = pos; b < stop; b += tile_blocks, ++t, s_off += s_step, r_off += r_step) {
                t->s_off = s_off;
                t->r_off = r_off;
                t->prec = gr.prec_id;
                t->sblk = blk + b;
                t->f = (int16_t)f;
                t->nblk = (int16_t)std::min(tile_blocks, stop - b);
                t->flags = 0;
            }
            const int made = (int)(t - (tiles + n_tiles));
            if (f > 0 && made > 0) {
                tiles[n_tiles].flags |= first_flag;
                last_idx = n_tiles + made - 1;
            }
            n_tiles += made;
            pos = stop;
        }
        k += gr.n_blocks;
        blk += gr.n_blocks;
    }
    close_range();
    wl.n_tiles = n_tiles;
    cta_begin[n_cta] = n_tiles;
}

extern "C" int32_t bf_schedule(const int32_t *f_of_slot, int32_t n_slots, const bf_group *groups, int32_t n_groups,
                               bf_precision prec, int32_t held, int32_t max_cta, bf_tile *tiles_out,
                               int32_t max_tiles, int32_t *cta_begin_out, int32_t *n_cta_out) {
    if (!f_of_slot || n_slots < 0 || n_groups < 0 || (n_groups && !groups) || max_cta < 1 || !n_cta_out ||
        prec < BF_FP32 || prec >= N_PREC || (held && !held_form(prec)))
        return -BF_EINVAL;
    for (int g = 0; g < n_groups; ++g) {
        if (groups[g].prec_id < 0 || groups[g].prec_id >= n_slots || groups[g].n_blocks < 0) return -BF_EINVAL;
        const int f = f_of_slot[groups[g].prec_id];
        if (f < 0 || f > F_LIMIT) return -BF_EINVAL;
    }
    static thread_local WorkList wl;  // reused: repeated calls allocate nothing
    const TuneTable tune;
    build_worklist(f_of_slot, tune, groups, n_groups, prec, held != 0, max_cta, R_BLOCK_BYTES, wl);
    const int nt = wl.n_tiles;
    *n_cta_out = (int32_t)wl.cta_begin.size() - 1;
    if (!tiles_out) return nt;  // size query
    if (nt > max_tiles || !cta_begin_out) return -BF_EINVAL;
    for (int t = 0; t < nt; ++t) {
        const Tile &a = wl.tiles[t];
        bf_tile &o = tiles_out[t];
        o.s_off = a.s_off;
        o.r_off = a.r_off;
        o.prec_id = a.prec;
        o.first_block = a.sblk;
        o.f = a.f;
        o.n_blocks = a.nblk;
        o.flags = a.flags;
    }
    for (size_t c = 0; c < wl.cta_begin.size(); ++c) cta_begin_out[c] = wl.cta_begin[c];
    return nt;
}

static bf_status validate_apply(bf_plan plan, const void *S, const float *scale, const bf_group *groups,
                                int32_t n_groups, bf_precision prec, const void *R, bool device_ptrs) {
    if (!plan) return bf_fail(nullptr, BF_EINVAL, "plan is NULL");
    if (n_groups < 0) return bf_fail(plan, BF_EINVAL, "negative n_groups");
    if (prec < BF_FP32 || prec >= N_PREC) return bf_fail(plan, BF_EINVAL, "unknown precision %d", (int)prec);
    if (scale && !held_form(prec))
        return bf_fail(plan, BF_EINVAL, "held S exists for BF_BF16, BF_FP16 and BF_BF16X3 only (scale_dev must be NULL)");
    if (n_groups == 0) return BF_OK;
    if (!groups || !S || !R) return bf_fail(plan, BF_EINVAL, "NULL argument");
    if (device_ptrs && (!aligned16(S) || !aligned16(R)))
        return bf_fail(plan, BF_EINVAL, "S_dev and R_dev must be 16-byte aligned");
    if (scale && ((uintptr_t)scale & 3u)) return bf_fail(plan, BF_EINVAL, "scale_dev must be 4-byte aligned");
    return check_group_slots(plan, groups, n_groups);
}

// Element size of R for an output type.
static int r_esize_of(int32_t rtype) { return rtype == BF_R_C64 ? 8 : 4; }
static int64_t r_block_stride_of(const bf_rlayout *layout) { return layout ? layout->block_stride : R_BLOCK_BYTES; }

static bf_status validate_rlayout(bf_plan plan, const bf_rlayout *l) {
    if (!l) return BF_OK;
    if (l->rtype < BF_R_C64 || l->rtype > BF_R_FP16) return bf_fail(plan, BF_EINVAL, "unknown R type %d", l->rtype);
    if (l->reserved != 0) return bf_fail(plan, BF_EINVAL, "bf_rlayout.reserved must be 0");
    const int64_t row_min = (int64_t)B_RE * r_esize_of(l->rtype);
    if (l->row_stride < row_min || l->block_stride < row_min || (l->row_stride & 15) || (l->block_stride & 15))
        return bf_fail(plan, BF_EINVAL, "R strides must be multiples of 16 and at least %lld bytes", (long long)row_min);
    return BF_OK;
}

static KParams make_params(bf_plan plan, const uint8_t *dlist, size_t tiles_bytes, const void *S, const float *scale,
                           void *R, bf_precision prec, const bf_rlayout *layout) {
    KParams p{};
    p.tiles = reinterpret_cast<const Tile *>(dlist);
    p.cta_begin = reinterpret_cast<const int32_t *>(dlist + tiles_bytes);
    p.S = (const uint8_t *)S;
    p.R = (uint8_t *)R;
    p.s_scale = scale;
    p.w_simt = plan->w_simt;
    p.w_tc = prec == BF_FP16 ? plan->w_fp16 : prec == BF_TF32X3 ? plan->w_tf32x2 : plan->w_bf16x2;
    p.w_tc_stride = prec == BF_FP16 ? W_FP16_STRIDE : prec == BF_TF32X3 ? W_TF32X2_STRIDE : W_BF16X2_STRIDE;
    p.w_scale = plan->w_scale;
    p.status = plan->d_status;
    p.r_row_stride = layout ? layout->row_stride : (int64_t)B_RE * 8;
    p.r_block_stride = r_block_stride_of(layout);
    p.r_type = layout ? layout->rtype : R_C64;
    p.r_esize = layout ? r_esize_of(layout->rtype) : 8;
    return p;
}

int max_cta_for(bf_plan plan, bf_precision prec) {
    const int g = prec == BF_FP32_3M ? 1 : 0;
    const int per_sm =
        simt_form(prec) ? std::max(1, std::min(plan->tune.simt_ctas_per_sm[g], plan->simt_resident[g])) : 1;
    return plan->sm_count * per_sm;
}

cudaError_t launch_kernel(bf_precision prec, bool held, const KParams &p, int n_cta, cudaStream_t st) {
    if (simt_form(prec)) return launch_simt(p, n_cta, st, prec == BF_FP32_3M);
    return launch_tc((int)prec, held, p, n_cta, st);
}

// Upload a work list through the plan's ring (one entry per call in flight)
// and launch it. `max_cta` <= 0 means the tuned default.
bf_status enqueue_apply(bf_plan plan, const void *S, const float *scale, const bf_group *groups, int32_t n_groups,
                        bf_precision prec, void *R, cudaStream_t st, int max_cta, const bf_rlayout *layout) {
    const bool held = scale != nullptr;
    WorkList &wl = plan->scratch_wl;
    build_worklist(plan->f_slot.data(), plan->tune, groups, n_groups, prec, held,
                   max_cta > 0 ? max_cta : max_cta_for(plan, prec), r_block_stride_of(layout), wl);
    if (wl.n_tiles == 0) return BF_OK;
    bf_status s;
    const size_t tb = (size_t)wl.n_tiles * sizeof(Tile), cb = wl.cta_begin.size() * sizeof(int32_t);
    const size_t bytes = tb + cb;
    // reuse an entry that already holds exactly this list
    WorkBuf *hit = nullptr;
    for (auto &w : plan->ring)
        if (w.valid && w.bytes == bytes && w.tiles_bytes == tb &&
            std::memcmp(w.h, wl.tiles.data(), tb) == 0 && std::memcmp(w.h + tb, wl.cta_begin.data(), cb) == 0) {
            hit = &w;
            break;
        }
    if (!hit) {
        WorkBuf &w = plan->ring[plan->ring_next];
        plan->ring_next = (plan->ring_next + 1) % (int)(sizeof(plan->ring) / sizeof(plan->ring[0]));
        BF_CK(plan, cudaEventSynchronize(w.ev));  // its previous launch has finished reading it
        w.valid = false;
        if ((s = grow_pinned(plan, &w.h, &w.hcap, bytes, true)) != BF_OK) return s;
        if ((s = grow_dev(plan, &w.d, &w.cap, bytes, true)) != BF_OK) return s;
        std::memcpy(w.h, wl.tiles.data(), tb);
        std::memcpy(w.h + tb, wl.cta_begin.data(), cb);
        BF_CK(plan, cudaMemcpyAsync(w.d, w.h, bytes, cudaMemcpyHostToDevice, st));
        w.bytes = bytes;
        w.tiles_bytes = tb;
        w.valid = true;
        hit = &w;
    } else {
        // the cached device copy may be in use on another stream: order after it
        BF_CK(plan, cudaStreamWaitEvent(st, hit->ev, 0));
    }
    const KParams p = make_params(plan, hit->d, tb, S, scale, R, prec, layout);
    BF_CK(plan, launch_kernel(prec, held, p, (int)wl.cta_begin.size() - 1, st));
    BF_CK(plan, cudaEventRecord(hit->ev, st));
    plan->launches++;
    return BF_OK;
}

extern "C" bf_status bf_apply_batch_rl(bf_plan plan, const void *S_dev, const float *scale_dev, const bf_group *groups,
                                       int32_t n_groups, bf_precision prec, void *R_dev, const bf_rlayout *layout,
                                       void *stream) {
    bf_status s = validate_apply(plan, S_dev, scale_dev, groups, n_groups, prec, R_dev, true);
    if (s == BF_OK) s = validate_rlayout(plan, layout);
    if (s != BF_OK || n_groups == 0) return s;
    if ((s = plan_ensure_device(plan)) != BF_OK) return s;
    return enqueue_apply(plan, S_dev, scale_dev, groups, n_groups, prec, R_dev, (cudaStream_t)stream, 0, layout);
}

extern "C" bf_status bf_apply_batch(bf_plan plan, const void *S_dev, const float *scale_dev, const bf_group *groups,
                                    int32_t n_groups, bf_precision prec, void *R_dev, void *stream) {
    return bf_apply_batch_rl(plan, S_dev, scale_dev, groups, n_groups, prec, R_dev, nullptr, stream);
}

// ------------------------------------------------------------------ prepared batches
struct bf_batch_s {
    bf_plan plan = nullptr;
    uint8_t *d = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    KParams p{};
    int n_cta = 0;
    bf_precision prec = BF_FP32;
    bool held = false;
};

extern "C" bf_status bf_batch_create_rl(bf_plan plan, const void *S_dev, const float *scale_dev,
                                        const bf_group *groups, int32_t n_groups, bf_precision prec, void *R_dev,
                                        const bf_rlayout *layout, bf_batch *out) {
    if (!out) return bf_fail(plan, BF_EINVAL, "out is NULL");
    *out = nullptr;
    bf_status s = validate_apply(plan, S_dev, scale_dev, groups, n_groups, prec, R_dev, true);
    if (s == BF_OK) s = validate_rlayout(plan, layout);
    if (s != BF_OK) return s;
    if ((s = plan_ensure_device(plan)) != BF_OK) return s;
    WorkList wl;
    build_worklist(plan->f_slot.data(), plan->tune, groups, n_groups, prec, scale_dev != nullptr,
                   max_cta_for(plan, prec), r_block_stride_of(layout), wl);
    bf_batch bt = new bf_batch_s();
    bt->plan = plan;
    const size_t tb = (size_t)wl.n_tiles * sizeof(Tile), cb = wl.cta_begin.size() * sizeof(int32_t);
    if (wl.n_tiles > 0) {
        if (cudaMalloc((void **)&bt->d, tb + cb) != cudaSuccess) {
            cudaGetLastError();
            delete bt;
            return bf_fail(plan, BF_ENOMEM, "work-list allocation failed");
        }
        cudaError_t e = cudaMemcpy(bt->d, wl.tiles.data(), tb, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(bt->d + tb, wl.cta_begin.data(), cb, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            bf_batch_destroy(bt);
            return bf_fail(plan, BF_ECUDA, "work-list upload: %s", cudaGetErrorString(e));
        }
    }
    bt->p = make_params(plan, bt->d, tb, S_dev, scale_dev, R_dev, prec, layout);
    bt->n_cta = wl.n_tiles == 0 ? 0 : (int)wl.cta_begin.size() - 1;
    bt->prec = prec;
    bt->held = scale_dev != nullptr;
    cudaError_t e = cudaStreamBeginCapture(plan->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess && bt->n_cta > 0) {
        cudaError_t le = launch_kernel(prec, bt->held, bt->p, bt->n_cta, plan->cap_stream);
        if (le != cudaSuccess) e = le;
    }
    cudaError_t ee = cudaStreamEndCapture(plan->cap_stream, &bt->graph);
    if (e == cudaSuccess) e = ee;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&bt->exec, bt->graph, 0);
    if (e != cudaSuccess) {
        cudaGetLastError();
        bf_batch_destroy(bt);
        return bf_fail(plan, BF_ECUDA, "graph capture: %s", cudaGetErrorString(e));
    }
    *out = bt;
    return BF_OK;
}

extern "C" bf_status bf_batch_create(bf_plan plan, const void *S_dev, const float *scale_dev, const bf_group *groups,
                                     int32_t n_groups, bf_precision prec, void *R_dev, bf_batch *out) {
    return bf_batch_create_rl(plan, S_dev, scale_dev, groups, n_groups, prec, R_dev, nullptr, out);
}

extern "C" bf_status bf_batch_launch(bf_batch batch, void *stream) {
    if (!batch) return bf_fail(nullptr, BF_EINVAL, "batch is NULL");
    bf_plan plan = batch->plan;
    if (batch->n_cta > 0) BF_CK(plan, launch_kernel(batch->prec, batch->held, batch->p, batch->n_cta, (cudaStream_t)stream));
    plan->launches++;
    return BF_OK;
}

extern "C" bf_status bf_batch_set_s_independent(bf_batch batch, int32_t independent) {
    if (!batch) return bf_fail(nullptr, BF_EINVAL, "batch is NULL");
    if (independent != 0 && independent != 1) return bf_fail(batch->plan, BF_EINVAL, "independent must be 0 or 1");
    batch->p.s_independent = independent;
    return BF_OK;
}

extern "C" bf_status bf_batch_launch_graph(bf_batch batch, void *stream) {
    if (!batch) return bf_fail(nullptr, BF_EINVAL, "batch is NULL");
    bf_plan plan = batch->plan;
    BF_CK(plan, cudaGraphLaunch(batch->exec, (cudaStream_t)stream));
    plan->launches++;
    return BF_OK;
}

extern "C" bf_status bf_batch_destroy(bf_batch batch) {
    if (!batch) return BF_OK;
    cudaSetDevice(batch->plan->device);
    if (batch->exec) cudaGraphExecDestroy(batch->exec);
    if (batch->graph) cudaGraphDestroy(batch->graph);
    if (batch->d) {
        cudaDeviceSynchronize();
        cudaFree(batch->d);
    }
    cudaGetLastError();
    delete batch;
    return BF_OK;
}

// ------------------------------------------------------------------ host buffers
// Chunks of consecutive groups flow through three streams: copy-in (x_in),
// compute (x_run) and copy-out (x_out), over a ring of BF_XFER_SLOTS device
// staging slots. Each direction of the host link stays busy on its own
// stream; a slot's S is reused once the kernel that read it has run, its R
// once the copy-out that read it has finished -- also across calls, so calls
// on different user streams pipeline through the three streams (the next
// call's copy-in runs while this one's copy-out finishes).
extern "C" bf_status bf_apply_batch_host(bf_plan plan, const void *S_host, const bf_group *groups, int32_t n_groups,
                                         bf_precision prec, void *R_host, void *stream) {
    bf_status s = validate_apply(plan, S_host, nullptr, groups, n_groups, prec, R_host, false);
    if (s != BF_OK || n_groups == 0) return s;
    if ((s = plan_ensure_device(plan)) != BF_OK) return s;
    cudaStream_t user = (cudaStream_t)stream;
    // chunking by bytes (S + R): the first chunk is small so that the
    // copy-out starts early, later ones double up to host_chunk_bytes (large
    // enough that issuing a chunk's calls takes less host time than the link
    // takes to move it)
    int64_t target = std::min<int64_t>(plan->host_chunk_first, plan->host_chunk_bytes);
    std::vector<int> cut{0};
    int64_t acc = 0, max_s = 0, max_r = 0, cs = 0, cr = 0;
    for (int g = 0; g < n_groups; ++g) {
        const int f = plan->f_slot[groups[g].prec_id];
        const int64_t sb = (int64_t)groups[g].n_blocks * f * S_BYTES_PER_F;
        const int64_t rb = (int64_t)groups[g].n_blocks * R_BLOCK_BYTES;
        if (acc > 0 && acc + sb + rb > target) {
            cut.push_back(g);
            target = std::min<int64_t>(2 * target, plan->host_chunk_bytes);
            max_s = std::max(max_s, cs);
            max_r = std::max(max_r, cr);
            acc = cs = cr = 0;
        }
        acc += sb + rb;
        cs += (sb + 15) & ~(int64_t)15;
        cr += rb;
    }
    cut.push_back(n_groups);
    max_s = std::max(max_s, cs);
    max_r = std::max(max_r, cr);
    const int n_chunks = (int)cut.size() - 1;
    // the slots this call will use, from the ring's current position
    for (int c = 0; c < std::min(n_chunks, BF_XFER_SLOTS); ++c) {
        const int i = (plan->x_next + c) % BF_XFER_SLOTS;
        if ((s = grow_dev(plan, &plan->x_s[i], &plan->x_scap[i], (size_t)std::max<int64_t>(max_s, 16))) != BF_OK) return s;
        if ((s = grow_dev(plan, &plan->x_r[i], &plan->x_rcap[i], (size_t)std::max<int64_t>(max_r, 16))) != BF_OK) return s;
    }
    BF_CK(plan, cudaEventRecord(plan->x_start, user));
    BF_CK(plan, cudaStreamWaitEvent(plan->x_in, plan->x_start, 0));
    BF_CK(plan, cudaStreamWaitEvent(plan->x_run, plan->x_start, 0));
    BF_CK(plan, cudaStreamWaitEvent(plan->x_out, plan->x_start, 0));
    std::vector<bf_group> local;
    for (int c = 0; c < n_chunks; ++c) {
        const int k = plan->x_next;
        plan->x_next = (plan->x_next + 1) % BF_XFER_SLOTS;
        // copy S in, merging groups that are contiguous in the host buffer,
        // once the last kernel that read this slot (this call's or an
        // earlier one's) has run
        BF_CK(plan, cudaStreamWaitEvent(plan->x_in, plan->x_run_done[k], 0));
        local.clear();
        int64_t so = 0, ro = 0;
        int64_t run_src = -1, run_dst = 0, run_len = 0;
        for (int g = cut[c]; g < cut[c + 1]; ++g) {
            const int f = plan->f_slot[groups[g].prec_id];
            const int64_t sb = (int64_t)groups[g].n_blocks * f * S_BYTES_PER_F;
            bf_group lg = groups[g];
            lg.s_off = so;
            lg.r_off = ro;
            local.push_back(lg);
            if (sb > 0) {
                if (run_src >= 0 && run_src + run_len == groups[g].s_off && run_dst + run_len == so) {
                    run_len += sb;
                } else {
                    if (run_len > 0)
                        BF_CK(plan, cudaMemcpyAsync(plan->x_s[k] + run_dst, (const uint8_t *)S_host + run_src, run_len,
                                                    cudaMemcpyHostToDevice, plan->x_in));
                    run_src = groups[g].s_off;
                    run_dst = so;
                    run_len = sb;
                }
            }
            so += (sb + 15) & ~(int64_t)15;
            ro += (int64_t)groups[g].n_blocks * R_BLOCK_BYTES;
        }
        if (run_len > 0)
            BF_CK(plan, cudaMemcpyAsync(plan->x_s[k] + run_dst, (const uint8_t *)S_host + run_src, run_len,
                                        cudaMemcpyHostToDevice, plan->x_in));
        BF_CK(plan, cudaEventRecord(plan->x_in_done[k], plan->x_in));
        // the product, once S is in and the slot's previous R has left
        BF_CK(plan, cudaStreamWaitEvent(plan->x_run, plan->x_in_done[k], 0));
        BF_CK(plan, cudaStreamWaitEvent(plan->x_run, plan->x_out_done[k], 0));
        if ((s = enqueue_apply(plan, plan->x_s[k], nullptr, local.data(), (int32_t)local.size(), prec, plan->x_r[k],
                               plan->x_run, 0)) != BF_OK)
            return s;
        BF_CK(plan, cudaEventRecord(plan->x_run_done[k], plan->x_run));
        // copy R out, merging contiguous destinations
        BF_CK(plan, cudaStreamWaitEvent(plan->x_out, plan->x_run_done[k], 0));
        int64_t rsrc = 0, rdst = -1, rlen = 0;
        for (int g = cut[c]; g < cut[c + 1]; ++g) {
            const int64_t rb = (int64_t)groups[g].n_blocks * R_BLOCK_BYTES;
            const int64_t lo = local[g - cut[c]].r_off;
            if (rb == 0) continue;
            if (rdst >= 0 && rdst + rlen == groups[g].r_off && rsrc + rlen == lo) {
                rlen += rb;
            } else {
                if (rlen > 0)
                    BF_CK(plan, cudaMemcpyAsync((uint8_t *)R_host + rdst, plan->x_r[k] + rsrc, rlen,
                                                cudaMemcpyDeviceToHost, plan->x_out));
                rsrc = lo;
                rdst = groups[g].r_off;
                rlen = rb;
            }
        }
        if (rlen > 0)
            BF_CK(plan, cudaMemcpyAsync((uint8_t *)R_host + rdst, plan->x_r[k] + rsrc, rlen, cudaMemcpyDeviceToHost,
                                        plan->x_out));
        BF_CK(plan, cudaEventRecord(plan->x_out_done[k], plan->x_out));
    }
    // every copy-in feeds a kernel and every kernel a copy-out, so the last
    // copy-out completes after all of this call's work
    BF_CK(plan, cudaEventRecord(plan->x_end, plan->x_out));
    BF_CK(plan, cudaStreamWaitEvent(user, plan->x_end, 0));
    return BF_OK;
}

// ------------------------------------------------------------------ accuracy report
extern "C" bf_status bf_errnorm(bf_plan plan, const void *R_dev, const void *Rref_dev, int64_t n_blocks,
                                double *per_block_dev, double *total_host, void *stream) {
    if (!plan) return bf_fail(nullptr, BF_EINVAL, "plan is NULL");
    if (n_blocks < 0 || !total_host) return bf_fail(plan, BF_EINVAL, "bad n_blocks or NULL total_host");
    if (n_blocks > 0 && (!R_dev || !Rref_dev)) return bf_fail(plan, BF_EINVAL, "NULL R_dev or Rref_dev");
    if ((R_dev && !aligned16(R_dev)) || (Rref_dev && !aligned16(Rref_dev)) ||
        (per_block_dev && ((uintptr_t)per_block_dev & 7u)))
        return bf_fail(plan, BF_EINVAL, "misaligned pointer");
    bf_status s = plan_ensure_device(plan);
    if (s != BF_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    double *pb = per_block_dev;
    const size_t need = ((size_t)(per_block_dev ? 0 : 2 * n_blocks) + 2) * sizeof(double);
    if ((s = grow_dev(plan, &plan->en_d, &plan->en_cap, need)) != BF_OK) return s;
    if ((s = grow_pinned(plan, &plan->en_h, &plan->en_hcap, 2 * sizeof(double))) != BF_OK) return s;
    double *total_dev = plan->en_d;
    if (!pb) pb = plan->en_d + 2;
    BF_CK(plan, launch_errnorm((const float2 *)R_dev, (const double2 *)Rref_dev, n_blocks, pb, total_dev,
                               plan->sm_count * 8, st));
    BF_CK(plan, cudaMemcpyAsync(plan->en_h, total_dev, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    BF_CK(plan, cudaStreamSynchronize(st));
    std::memcpy(total_host, plan->en_h, 2 * sizeof(double));
    return BF_OK;
}

extern "C" int64_t bf_plan_launch_count(bf_plan plan) { return plan ? plan->launches : 0; }
