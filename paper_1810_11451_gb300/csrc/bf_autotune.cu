// bf_autotune.cu -- the project's autotuner: per precision and f bucket it
// times the product on synthetic batches of two sizes on this GPU, takes the
// slope (marginal ns per block) as the scheduling cost, and keeps the tile
// size (1 or 2 blocks per tile) that ran faster. The paper's optimizer picks,
// per matrix size and target, the best building block for an operation
// (Sec. IV); this picks, per f and GPU, the launch shape of one kernel and
// the costs that balance uneven batches across CTAs.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "bf_internal.h"
#include "bf_plan.h"

using namespace bfi;

namespace {

constexpr int SLOTS_PER_F = 16;  // distinct precoders per bucket, so W is reloaded as in real batches
constexpr int GROUP_BLOCKS = 14;
constexpr int REPS = 9, WARM = 3;

struct Scratch {
    uint8_t *W = nullptr, *S = nullptr, *R = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    ~Scratch() {
        if (W) cudaFree(W);
        if (S) cudaFree(S);
        if (R) cudaFree(R);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        cudaGetLastError();
    }
};

bf_status time_batch(bf_plan plan, const Scratch &sc, bf_precision prec, int f, int slot0, int n_blocks,
                     cudaStream_t st, double *ms_out) {
    std::vector<bf_group> groups;
    const int64_t sb = (int64_t)f * S_BYTES_PER_F;
    for (int b = 0, g = 0; b < n_blocks; b += GROUP_BLOCKS, ++g) {
        bf_group gr;
        gr.prec_id = slot0 + g % SLOTS_PER_F;
        gr.n_blocks = std::min(GROUP_BLOCKS, n_blocks - b);
        gr.s_off = (int64_t)b * sb;
        gr.r_off = (int64_t)b * R_BLOCK_BYTES;
        groups.push_back(gr);
    }
    std::vector<float> t;
    for (int r = 0; r < WARM + REPS; ++r) {
        if (cudaEventRecord(sc.e0, st) != cudaSuccess) return bf_fail(plan, BF_ECUDA, "cudaEventRecord");
        bf_status s = enqueue_apply(plan, sc.S, nullptr, groups.data(), (int32_t)groups.size(), prec, sc.R, st, 0);
        if (s != BF_OK) return s;
        if (cudaEventRecord(sc.e1, st) != cudaSuccess || cudaEventSynchronize(sc.e1) != cudaSuccess)
            return bf_fail(plan, BF_ECUDA, "timing event");
        float ms = 0.f;
        cudaEventElapsedTime(&ms, sc.e0, sc.e1);
        if (r >= WARM) t.push_back(ms);
    }
    std::sort(t.begin(), t.end());
    *ms_out = t[t.size() / 2];
    return BF_OK;
}

}  // namespace

extern "C" bf_status bf_autotune(bf_plan plan, bf_precision prec, void *stream) {
    if (!plan) return bf_fail(nullptr, BF_EINVAL, "plan is NULL");
    if (prec < BF_FP32 || prec >= N_PREC) return bf_fail(plan, BF_EINVAL, "unknown precision");
    bf_status s = plan_ensure_device(plan);
    if (s != BF_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    const int n1 = plan->sm_count * 8, n2 = plan->sm_count * 32;  // blocks
    Scratch sc;
    const size_t wbytes = (size_t)SLOTS_PER_F * N_ANT * F_LIMIT * 8;
    if (cudaMalloc((void **)&sc.W, wbytes) != cudaSuccess ||
        cudaMalloc((void **)&sc.S, (size_t)n2 * F_LIMIT * S_BYTES_PER_F) != cudaSuccess ||
        cudaMalloc((void **)&sc.R, (size_t)n2 * R_BLOCK_BYTES) != cudaSuccess ||
        cudaEventCreate(&sc.e0) != cudaSuccess || cudaEventCreate(&sc.e1) != cudaSuccess) {
        cudaGetLastError();
        return bf_fail(plan, BF_ENOMEM, "autotune scratch allocation failed");
    }
    // Finite, non-trivial values (0x3C3C3C3C is about 0.0115 as an FP32).
    if (cudaMemsetAsync(sc.W, 0x3C, wbytes, st) != cudaSuccess ||
        cudaMemsetAsync(sc.S, 0x3C, (size_t)n2 * F_LIMIT * S_BYTES_PER_F, st) != cudaSuccess)
        return bf_fail(plan, BF_ECUDA, "autotune scratch fill failed");
    // Temporary precoder slots above every slot in use: SLOTS_PER_F per bucket.
    const int base = plan->cap;
    std::vector<int32_t> fs;
    for (int b = 0; b < TUNE_BUCKETS; ++b)
        for (int k = 0; k < SLOTS_PER_F; ++k) fs.push_back(std::min(TUNE_REP_F[b], plan->f_max));
    for (int b = 0; b < TUNE_BUCKETS; ++b)
        if ((s = bf_set_precoders(plan, sc.W, fs.data() + b * SLOTS_PER_F, SLOTS_PER_F, base + b * SLOTS_PER_F,
                                  stream)) != BF_OK)
            return s;

    TuneTable &T = plan->tune;
    const int p = (int)prec;
    T.tuned[p] = false;  // measure under the byte-based split
    bf_status result = BF_OK;
    for (int b = 0; b < TUNE_BUCKETS && result == BF_OK; ++b) {
        const int f = fs[b * SLOTS_PER_F];
        double best_t2 = 1e30, best_slope = 0.0;
        int best_tb = 2;
        for (int tb = 1; tb <= 2; ++tb) {
            T.tile_blocks[p][b] = tb;
            double t1 = 0, t2 = 0;
            if ((result = time_batch(plan, sc, prec, f, base + b * SLOTS_PER_F, n1, st, &t1)) != BF_OK) break;
            if ((result = time_batch(plan, sc, prec, f, base + b * SLOTS_PER_F, n2, st, &t2)) != BF_OK) break;
            if (t2 < best_t2) {
                best_t2 = t2;
                best_tb = tb;
                best_slope = std::max(1e-3, (t2 - t1) * 1e6 / (n2 - n1));  // ns per block
            }
        }
        T.tile_blocks[p][b] = best_tb;
        T.ns_per_block[p][b] = best_slope;
    }
    if (result == BF_OK && simt_form(prec)) {
        // CTAs per SM of this CUDA-core kernel, at f = 36
        const int g = prec == BF_FP32_3M ? 1 : 0;
        double best = 1e30;
        int best_c = T.simt_ctas_per_sm[g];
        for (int c = 1; c <= plan->simt_resident[g]; ++c) {
            T.simt_ctas_per_sm[g] = c;
            double t2 = 0;
            if ((result = time_batch(plan, sc, prec, fs[(TUNE_BUCKETS - 1) * SLOTS_PER_F],
                                     base + (TUNE_BUCKETS - 1) * SLOTS_PER_F, n2, st, &t2)) != BF_OK)
                break;
            if (t2 < best) {
                best = t2;
                best_c = c;
            }
        }
        T.simt_ctas_per_sm[g] = best_c;
    }
    if (cudaStreamSynchronize(st) != cudaSuccess) result = bf_fail(plan, BF_ECUDA, "autotune synchronize");
    for (int i = 0; i < TUNE_BUCKETS * SLOTS_PER_F; ++i) plan->f_slot[base + i] = -1;  // release the slots
    if (result == BF_OK) T.tuned[p] = true;
    return result;
}

extern "C" bf_status bf_tune_query(bf_plan plan, bf_precision prec, int32_t f, double *ns_per_block,
                                   int32_t *tile_blocks, int32_t *tuned) {
    if (!plan || prec < BF_FP32 || prec >= N_PREC || f < 0 || f > F_LIMIT)
        return bf_fail(plan, BF_EINVAL, "bad arguments");
    const TuneTable &T = plan->tune;
    if (ns_per_block) *ns_per_block = T.ns_per_block[prec][f_bucket(f)];
    if (tile_blocks) *tile_blocks = T.tile_blocks[prec][f_bucket(f)];
    if (tuned) *tuned = T.tuned[prec] ? 1 : 0;
    return BF_OK;
}

extern "C" bf_status bf_tune_save(bf_plan plan, const char *path) {
    if (!plan || !path) return bf_fail(plan, BF_EINVAL, "NULL argument");
    FILE *fh = fopen(path, "w");
    if (!fh) return bf_fail(plan, BF_EINVAL, "cannot open %s for writing", path);
    const TuneTable &T = plan->tune;
    std::string name = plan->device_name;
    for (char &ch : name)
        if (ch == '"' || ch == '\\' || (unsigned char)ch < 0x20) ch = '_';
    fprintf(fh, "{\n  \"format\": \"libbf-tune-2\",\n  \"kind\": \"product\",\n");
    fprintf(fh, "  \"target\": {\"device\": \"%s\", \"cc\": %d, \"sm_count\": %d},\n", name.c_str(), plan->cc,
            plan->sm_count);
    fprintf(fh, "  \"simt_ctas_per_sm\": [%d, %d],\n", T.simt_ctas_per_sm[0], T.simt_ctas_per_sm[1]);
    fprintf(fh, "  \"f_bucket_upper\": [0, 8, 16, 24, 36],\n  \"precisions\": [\n");
    for (int p = 0; p < N_PREC; ++p) {
        fprintf(fh, "    {\"precision\": %d, \"tuned\": %d, \"ns_per_block\": [", p, T.tuned[p] ? 1 : 0);
        for (int b = 0; b < TUNE_BUCKETS; ++b) fprintf(fh, "%s%.6f", b ? ", " : "", T.ns_per_block[p][b]);
        fprintf(fh, "], \"tile_blocks\": [");
        for (int b = 0; b < TUNE_BUCKETS; ++b) fprintf(fh, "%s%d", b ? ", " : "", T.tile_blocks[p][b]);
        fprintf(fh, "]}%s\n", p < N_PREC - 1 ? "," : "");
    }
    fprintf(fh, "  ]\n}\n");
    const bool ok = fclose(fh) == 0;
    return ok ? BF_OK : bf_fail(plan, BF_EINVAL, "write to %s failed", path);
}

namespace {

bool read_file(const char *path, std::string &txt) {
    FILE *fh = fopen(path, "r");
    if (!fh) return false;
    char buf[4096];
    size_t n;
    while ((n = fread(buf, 1, sizeof buf, fh)) > 0) txt.append(buf, n);
    fclose(fh);
    return true;
}

// The target a table was measured on: the "target" object bf_tune_save writes.
bool parse_target(const std::string &txt, std::string &name, int &cc, int &sms) {
    static const char key[] = "\"target\": {\"device\": \"";
    size_t pos = txt.find(key);
    if (pos == std::string::npos) return false;
    pos += sizeof key - 1;
    const size_t end = txt.find('"', pos);
    if (end == std::string::npos) return false;
    name = txt.substr(pos, end - pos);
    return sscanf(txt.c_str() + end, "\", \"cc\": %d, \"sm_count\": %d}", &cc, &sms) == 2;
}

// BF_OK when the table at `txt` was measured on this target, else BF_EINVAL
// with the reason (errors are reported on `plan`, which may be NULL).
bf_status check_target(bf_plan plan, const char *path, const std::string &txt, const char *device, int cc,
                       int sm_count) {
    if (txt.find("\"libbf-tune-2\"") == std::string::npos)
        return bf_fail(plan, BF_EINVAL, "%s: not a libbf tune table with a recorded target (libbf-tune-2)", path);
    std::string name;
    int tcc = 0, tsms = 0;
    if (!parse_target(txt, name, tcc, tsms)) return bf_fail(plan, BF_EINVAL, "%s: unreadable target", path);
    if (name != device || tcc != cc || tsms != sm_count)
        return bf_fail(plan, BF_EINVAL,
                       "%s: measured on \"%s\" (sm_%d, %d SMs), not on this target \"%s\" (sm_%d, %d SMs)", path,
                       name.c_str(), tcc, tsms, device, cc, sm_count);
    return BF_OK;
}

}  // namespace

extern "C" bf_status bf_tune_check_target(const char *path, const char *device_name, int32_t cc,
                                          int32_t sm_count) {
    if (!path || !device_name) return bf_fail(nullptr, BF_EINVAL, "NULL argument");
    std::string txt;
    if (!read_file(path, txt)) return bf_fail(nullptr, BF_EINVAL, "cannot open %s", path);
    return check_target(nullptr, path, txt, device_name, cc, sm_count);
}

// Reads the format bf_tune_save writes (keys in that order), after checking
// that it was measured on this plan's device.
extern "C" bf_status bf_tune_load(bf_plan plan, const char *path) {
    if (!plan || !path) return bf_fail(plan, BF_EINVAL, "NULL argument");
    std::string txt;
    if (!read_file(path, txt)) return bf_fail(plan, BF_EINVAL, "cannot open %s", path);
    auto bad = [&](const char *why) { return bf_fail(plan, BF_EINVAL, "%s: %s", path, why); };
    bf_status ts = check_target(plan, path, txt, plan->device_name.c_str(), plan->cc, plan->sm_count);
    if (ts != BF_OK) return ts;
    if (txt.find("\"kind\": \"filter\"") != std::string::npos) return bad("a filter tune table, not a product one");
    size_t pos;
    TuneTable T;
    pos = txt.find("\"simt_ctas_per_sm\": [");
    if (pos == std::string::npos ||
        sscanf(txt.c_str() + pos + 21, "%d, %d", &T.simt_ctas_per_sm[0], &T.simt_ctas_per_sm[1]) != 2 ||
        T.simt_ctas_per_sm[0] < 1 || T.simt_ctas_per_sm[0] > 16 || T.simt_ctas_per_sm[1] < 1 ||
        T.simt_ctas_per_sm[1] > 16)
        return bad("simt_ctas_per_sm");
    for (int p = 0; p < N_PREC; ++p) {
        char key[32];
        snprintf(key, sizeof key, "\"precision\": %d,", p);
        pos = txt.find(key);
        if (pos == std::string::npos) return bad("missing precision");
        int tuned = 0;
        size_t q = txt.find("\"tuned\":", pos);
        if (q == std::string::npos || sscanf(txt.c_str() + q + 8, "%d", &tuned) != 1) return bad("tuned");
        T.tuned[p] = tuned != 0;
        q = txt.find("\"ns_per_block\": [", pos);
        if (q == std::string::npos) return bad("ns_per_block");
        const char *c = txt.c_str() + q + 17;
        for (int b = 0; b < TUNE_BUCKETS; ++b) {
            char *end = nullptr;
            T.ns_per_block[p][b] = strtod(c, &end);
            if (end == c || T.ns_per_block[p][b] < 0) return bad("ns_per_block value");
            c = end + (*end == ',' ? 1 : 0);
        }
        q = txt.find("\"tile_blocks\": [", pos);
        if (q == std::string::npos) return bad("tile_blocks");
        c = txt.c_str() + q + 16;
        for (int b = 0; b < TUNE_BUCKETS; ++b) {
            char *end = nullptr;
            const long v = strtol(c, &end, 10);
            if (end == c || (v != 1 && v != 2)) return bad("tile_blocks value");
            T.tile_blocks[p][b] = (int)v;
            c = end + (*end == ',' ? 1 : 0);
        }
    }
    plan->tune = T;
    return BF_OK;
}

extern "C" bf_status bf_select_form(bf_plan plan, bf_target target, const bf_group *groups, int32_t n_groups,
                                    bf_precision *prec_out, double *ns_out) {
    if (!plan || !prec_out || n_groups < 0 || (n_groups > 0 && !groups) ||
        (target != BF_TARGET_FP32 && target != BF_TARGET_BF16))
        return bf_fail(plan, BF_EINVAL, "bad arguments");
    for (int g = 0; g < n_groups; ++g)
        if (groups[g].n_blocks < 0 || groups[g].prec_id < 0 || groups[g].prec_id >= plan->cap ||
            plan->f_slot[groups[g].prec_id] < 0)
            return bf_fail(plan, BF_ENOTFOUND, "group %d: precoder slot %d is not set", g, groups[g].prec_id);
    static const bf_precision fp32_forms[] = {BF_BF16X3, BF_TF32X3, BF_FP32, BF_FP32_3M};
    static const bf_precision all_forms[] = {BF_BF16, BF_FP16, BF_BF16X3, BF_TF32X3, BF_FP32, BF_FP32_3M};
    const bf_precision *cand = target == BF_TARGET_FP32 ? fp32_forms : all_forms;
    const int n_cand = target == BF_TARGET_FP32 ? 4 : 6;
    const TuneTable &T = plan->tune;
    bf_precision best = cand[0];
    double best_ns = -1.0;
    for (int i = 0; i < n_cand; ++i) {
        const int p = (int)cand[i];
        if (!T.tuned[p]) continue;
        double ns = 0.0;
        for (int g = 0; g < n_groups; ++g)
            ns += (double)groups[g].n_blocks * T.ns_per_block[p][f_bucket(plan->f_slot[groups[g].prec_id])];
        if (best_ns < 0 || ns < best_ns) {
            best_ns = ns;
            best = cand[i];
        }
    }
    *prec_out = best;
    if (ns_out) *ns_out = best_ns < 0 ? 0.0 : best_ns;
    return BF_OK;
}
