// bf_serve.cu -- the continuous-batching serving loop of include/bf_serve.h:
// FIFO queue, HBM-budget admission, launch slots (one stream each), merged
// launches of the persistent product kernel, completion by event polling, a
// watchdog on launches that do not complete and per-job deadline accounting.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "bf_internal.h"
#include "bf_plan.h"
#include "bf_serve.h"

using namespace bfi;

namespace {

enum JobState { QUEUED = 0, RUNNING = 1, DONE = 2 };

struct JobRec {
    int cell = 0;
    bf_precision prec = BF_FP32;
    std::vector<bf_group> groups;  // absolute byte addresses in s_off / r_off
    int32_t slot_lo = 0, slot_hi = 0;  // precoder slots read: [slot_lo, slot_hi)
    int64_t bytes = 0;
    int64_t arrival_ns = 0;
    int64_t submit_ns = 0, admit_ns = 0, launched_ns = 0;
    int64_t done_ns = 0;
    int state = QUEUED;
    bool waited_budget = false;
    bf_status status = BF_OK;
};

struct Slot {
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    bool busy = false;
    int64_t fake_done_ns = 0;
    int64_t launched_ns = 0;   // when the launch was enqueued (the watchdog's start)
    bool timed_out = false;    // the watchdog failed its jobs; the launch still runs
    int64_t held_bytes = 0;    // budget of those jobs, released when it completes
    std::vector<uint64_t> jobs;
};

// A precoder conversion that later launches reading its slots must follow.
struct PrepRec {
    int32_t lo, hi;  // slots [lo, hi)
    cudaEvent_t ev;
};

}  // namespace

struct bf_server_s {
    bf_plan plan = nullptr;
    bf_serve_config cfg{};
    bool fake = false;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<uint64_t> queue;
    std::unordered_map<uint64_t, JobRec> jobs;
    std::vector<Slot> slots;
    int64_t inflight_bytes = 0;
    uint64_t next_ticket = 1;
    bool stop = false, paused = false, exited = false;
    std::thread th;
    bf_serve_stats stats{};
    std::mutex plan_mu;  // the plan is used by the dispatcher and bf_serve_set_precoders
    // the plan's precoder-slot table, read by bf_submit; bf_serve_set_precoders
    // holds it (inside plan_mu) while it changes the table, so submitters
    // never wait behind a launch
    std::mutex slot_mu;
    cudaStream_t prep_st = nullptr;
    std::vector<PrepRec> prep_pending;  // conversions not yet seen complete (under plan_mu)
    std::vector<cudaEvent_t> prep_pool;  // their spare events
    std::vector<bf_group> merged;
    std::vector<std::pair<int32_t, int32_t>> merged_slots;  // slot ranges of the merged jobs
};

// A job leaves the engine (completed, failed or timed out): its latency is
// accounted against the deadline and the worst job's breakdown kept.
static void account_done(bf_server_s *srv, JobRec &j) {
    const int64_t lat = j.done_ns - j.arrival_ns;
    const int64_t part[4] = {j.submit_ns - j.arrival_ns,
                             j.admit_ns ? j.admit_ns - j.submit_ns : j.done_ns - j.submit_ns,
                             j.launched_ns && j.admit_ns ? j.launched_ns - j.admit_ns : 0,
                             j.launched_ns ? j.done_ns - j.launched_ns : 0};
    bf_serve_stats &st = srv->stats;
    st.sum_submit_ns += part[0];
    st.sum_queue_ns += part[1];
    st.sum_launch_ns += part[2];
    st.sum_device_ns += part[3];
    if (lat > st.deadline_ns) {
        st.over_deadline++;
        const int k = (int)(std::max_element(part, part + 4) - part);
        int64_t *by[4] = {&st.over_by_submit, &st.over_by_queue, &st.over_by_launch, &st.over_by_device};
        ++*by[k];
    }
    if (lat > st.worst_latency_ns) {
        st.worst_latency_ns = lat;
        st.worst_submit_ns = part[0];
        st.worst_queue_ns = part[1];
        st.worst_launch_ns = part[2];
        st.worst_device_ns = part[3];
    }
}

extern "C" int64_t bf_now_ns(void) {
    return std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

static int64_t job_bytes(const int *f_slot, const bf_job *job) {
    int64_t b = 0;
    for (int g = 0; g < job->n_groups; ++g) {
        const int f = f_slot ? f_slot[job->groups[g].prec_id] : 0;
        b += (int64_t)job->groups[g].n_blocks * ((int64_t)f * S_BYTES_PER_F + R_BLOCK_BYTES);
    }
    return b;
}

// Launch one merged batch on a slot (called without the queue lock). The
// launch follows every pending precoder conversion whose slots one of its
// jobs reads, and no other: a cell's next-epoch update does not hold back the
// other cells' jobs.
static bf_status launch_slot(bf_server srv, Slot &slot, bf_precision prec, const std::vector<bf_group> &groups,
                             const std::vector<std::pair<int32_t, int32_t>> &slot_ranges) {
    if (srv->fake) {
        slot.fake_done_ns = bf_now_ns() + (int64_t)srv->cfg.fake_device_us * 1000;
        return BF_OK;
    }
    std::lock_guard<std::mutex> pl(srv->plan_mu);
    bf_plan plan = srv->plan;
    for (size_t i = 0; i < srv->prep_pending.size();) {
        PrepRec &r = srv->prep_pending[i];
        const cudaError_t e = cudaEventQuery(r.ev);
        if (e == cudaSuccess) {  // complete: nothing to order after
            srv->prep_pool.push_back(r.ev);
            r = srv->prep_pending.back();
            srv->prep_pending.pop_back();
            continue;
        }
        if (e != cudaErrorNotReady) return bf_fail(plan, BF_ECUDA, "cudaEventQuery: %s", cudaGetErrorString(e));
        bool reads = false;
        for (const auto &sr : slot_ranges) reads = reads || (sr.first < r.hi && r.lo < sr.second);
        if (reads && cudaStreamWaitEvent(slot.st, r.ev, 0) != cudaSuccess)
            return bf_fail(plan, BF_ECUDA, "cudaStreamWaitEvent failed");
        ++i;
    }
    // S and R bases are 0: the groups carry absolute device addresses, so jobs
    // with different buffers share one launch.
    bf_status s = enqueue_apply(plan, nullptr, nullptr, groups.data(), (int32_t)groups.size(), prec, nullptr,
                                slot.st, 0);
    if (s != BF_OK) return s;
    if (cudaEventRecord(slot.ev, slot.st) != cudaSuccess) return bf_fail(plan, BF_ECUDA, "cudaEventRecord failed");
    return BF_OK;
}

static void dispatcher(bf_server srv) {
    // Only this thread changes the slots, so their events are queried without
    // the queue lock; submitters never wait behind a poll.
    std::vector<int> busy_idx;
    std::vector<char> done_flag;
    std::vector<bf_status> done_st;
    std::unique_lock<std::mutex> lk(srv->mu);
    for (;;) {
        bool any_busy = false, progressed = false;
        // 1. completions
        busy_idx.clear();
        for (int i = 0; i < (int)srv->slots.size(); ++i)
            if (srv->slots[i].busy) busy_idx.push_back(i);
        lk.unlock();
        done_flag.assign(busy_idx.size(), 0);
        done_st.assign(busy_idx.size(), BF_OK);
        const int64_t t_query = bf_now_ns();
        for (size_t k = 0; k < busy_idx.size(); ++k) {
            const Slot &sl = srv->slots[busy_idx[k]];
            if (srv->fake) {
                done_flag[k] = t_query >= sl.fake_done_ns;
            } else {
                const cudaError_t e = cudaEventQuery(sl.ev);
                done_flag[k] = e != cudaErrorNotReady;
                if (done_flag[k] && e != cudaSuccess) done_st[k] = BF_ECUDA;
            }
        }
        const int64_t now = bf_now_ns();
        lk.lock();
        for (size_t k = 0; k < busy_idx.size(); ++k) {
            Slot &sl = srv->slots[busy_idx[k]];
            const bf_status st = done_st[k];
            if (!done_flag[k]) {
                any_busy = true;
                // watchdog: give the launch's jobs up, keep the slot and their
                // budget until the device is done with their buffers
                if (!sl.timed_out && now - sl.launched_ns > srv->stats.slot_timeout_ns) {
                    for (uint64_t t : sl.jobs) {
                        JobRec &j = srv->jobs[t];
                        j.state = DONE;
                        j.status = BF_ETIMEOUT;
                        j.done_ns = now;
                        sl.held_bytes += j.bytes;
                        srv->stats.completed++;
                        srv->stats.timed_out++;
                        account_done(srv, j);
                    }
                    sl.jobs.clear();
                    sl.timed_out = true;
                    progressed = true;
                    srv->cv_done.notify_all();
                }
                continue;
            }
            if (sl.timed_out) {  // a given-up launch finally completed
                srv->inflight_bytes -= sl.held_bytes;
                sl.held_bytes = 0;
                sl.timed_out = false;
            }
            for (uint64_t t : sl.jobs) {
                JobRec &j = srv->jobs[t];
                j.state = DONE;
                j.status = st;
                j.done_ns = now;
                srv->inflight_bytes -= j.bytes;
                srv->stats.completed++;
                account_done(srv, j);
            }
            sl.jobs.clear();
            sl.busy = false;
            progressed = true;
            srv->cv_done.notify_all();
        }
        // 2. admission: FIFO, one precision per launch, within the budget
        while (!srv->paused && !srv->queue.empty()) {
            Slot *free_slot = nullptr;
            for (Slot &sl : srv->slots)
                if (!sl.busy) {
                    free_slot = &sl;
                    break;
                }
            if (!free_slot) break;
            JobRec &head = srv->jobs[srv->queue.front()];
            if (srv->inflight_bytes + head.bytes > srv->cfg.hbm_budget_bytes) {
                if (!head.waited_budget) {
                    head.waited_budget = true;
                    srv->stats.budget_waits++;
                }
                break;
            }
            const bf_precision prec = head.prec;
            std::vector<uint64_t> take;
            int64_t add = 0;
            while (!srv->queue.empty() && (int)take.size() < srv->cfg.max_batch_jobs) {
                JobRec &j = srv->jobs[srv->queue.front()];
                if (j.prec != prec || srv->inflight_bytes + add + j.bytes > srv->cfg.hbm_budget_bytes) break;
                take.push_back(srv->queue.front());
                add += j.bytes;
                srv->queue.pop_front();
            }
            srv->merged.clear();
            srv->merged_slots.clear();
            const int64_t t_admit = bf_now_ns();
            for (uint64_t t : take) {
                JobRec &j = srv->jobs[t];
                j.state = RUNNING;
                j.admit_ns = t_admit;
                srv->merged.insert(srv->merged.end(), j.groups.begin(), j.groups.end());
                srv->merged_slots.emplace_back(j.slot_lo, j.slot_hi);
            }
            srv->inflight_bytes += add;
            srv->stats.max_inflight_bytes = std::max(srv->stats.max_inflight_bytes, srv->inflight_bytes);
            free_slot->busy = true;
            free_slot->jobs = take;
            std::vector<bf_group> groups;
            groups.swap(srv->merged);
            std::vector<std::pair<int32_t, int32_t>> ranges;
            ranges.swap(srv->merged_slots);
            lk.unlock();
            const bf_status st = launch_slot(srv, *free_slot, prec, groups, ranges);
            const int64_t t_launched = bf_now_ns();
            lk.lock();
            free_slot->launched_ns = t_launched;
            for (uint64_t t : take) srv->jobs[t].launched_ns = t_launched;
            srv->stats.launches++;
            srv->stats.max_jobs_per_launch = std::max(srv->stats.max_jobs_per_launch, (int32_t)take.size());
            int busy = 0;
            for (Slot &sl : srv->slots) busy += sl.busy ? 1 : 0;
            srv->stats.max_busy_slots = std::max(srv->stats.max_busy_slots, busy);
            if (st != BF_OK) {  // the launch failed: complete its jobs with the error
                for (uint64_t t : take) {
                    JobRec &j = srv->jobs[t];
                    j.state = DONE;
                    j.status = st;
                    j.done_ns = bf_now_ns();
                    srv->inflight_bytes -= j.bytes;
                    srv->stats.completed++;
                    account_done(srv, j);
                }
                free_slot->jobs.clear();
                free_slot->busy = false;
                srv->cv_done.notify_all();
            }
            any_busy = true;
            progressed = true;
        }
        if (srv->stop && srv->queue.empty() && !any_busy) break;
        if (!any_busy && (srv->queue.empty() || srv->paused)) {
            srv->cv_work.wait_for(lk, std::chrono::milliseconds(2));
        } else if (!progressed) {
            // launches in flight: keep polling, giving the core away between polls
            lk.unlock();
            std::this_thread::yield();
            lk.lock();
        }
    }
    srv->exited = true;
    srv->cv_done.notify_all();
}

extern "C" bf_status bf_serve_create(bf_plan plan, const bf_serve_config *cfg, bf_server *out) {
    if (!out || !cfg) return bf_fail(plan, BF_EINVAL, "NULL argument");
    *out = nullptr;
    if (cfg->n_slots < 1 || cfg->n_slots > 8 || cfg->max_batch_jobs < 1 || cfg->queue_capacity < 1 ||
        cfg->hbm_budget_bytes <= 0 || cfg->fake_device_us < 0 || cfg->deadline_us < 0 || cfg->slot_timeout_us < 0)
        return bf_fail(plan, BF_EINVAL, "bad serving configuration");
    if (!plan && cfg->fake_device_us == 0) return bf_fail(nullptr, BF_EINVAL, "plan is NULL");
    bf_server s = new bf_server_s();
    s->plan = plan;
    s->cfg = *cfg;
    s->fake = cfg->fake_device_us > 0;
    s->stats.deadline_ns = (int64_t)(cfg->deadline_us ? cfg->deadline_us : 500) * 1000;
    s->stats.slot_timeout_ns = (int64_t)(cfg->slot_timeout_us ? cfg->slot_timeout_us : 50000) * 1000;
    s->slots.resize(cfg->n_slots);
    if (!s->fake) {
        bf_status st = plan_ensure_device(plan);
        if (st != BF_OK) {
            delete s;
            return st;
        }
        bool ok = cudaStreamCreateWithFlags(&s->prep_st, cudaStreamNonBlocking) == cudaSuccess;
        for (Slot &sl : s->slots)
            ok = ok && cudaStreamCreateWithFlags(&sl.st, cudaStreamNonBlocking) == cudaSuccess &&
                 cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming) == cudaSuccess;
        if (!ok) {
            cudaGetLastError();
            for (Slot &sl : s->slots) {
                if (sl.st) cudaStreamDestroy(sl.st);
                if (sl.ev) cudaEventDestroy(sl.ev);
            }
            if (s->prep_st) cudaStreamDestroy(s->prep_st);
            delete s;
            return bf_fail(plan, BF_ECUDA, "stream/event creation failed");
        }
    }
    s->th = std::thread(dispatcher, s);
    if (plan) plan->servers++;
    *out = s;
    return BF_OK;
}

extern "C" bf_status bf_serve_destroy(bf_server srv, int64_t timeout_us) {
    if (!srv) return BF_OK;
    {
        std::unique_lock<std::mutex> lk(srv->mu);
        srv->stop = true;
        srv->cv_work.notify_all();
        const auto deadline = std::chrono::steady_clock::now() + std::chrono::microseconds(std::max<int64_t>(0, timeout_us));
        if (!srv->cv_done.wait_until(lk, deadline, [&] { return srv->exited; })) {
            srv->stop = false;  // keep serving; the caller may resume and retry
            return bf_fail(srv->plan, BF_EBUSY, "server still has queued or running jobs");
        }
    }
    srv->th.join();
    if (!srv->fake) {
        for (Slot &sl : srv->slots) {
            cudaStreamSynchronize(sl.st);
            cudaStreamDestroy(sl.st);
            cudaEventDestroy(sl.ev);
        }
        cudaStreamSynchronize(srv->prep_st);
        cudaStreamDestroy(srv->prep_st);
        for (const PrepRec &r : srv->prep_pending) cudaEventDestroy(r.ev);
        for (cudaEvent_t e : srv->prep_pool) cudaEventDestroy(e);
        cudaGetLastError();
    }
    if (srv->plan) srv->plan->servers--;
    delete srv;
    return BF_OK;
}

extern "C" bf_status bf_serve_set_precoders(bf_server srv, const void *W_dev, const int32_t *f_host, int32_t n_prec,
                                            int32_t first_id) {
    if (!srv) return bf_fail(nullptr, BF_EINVAL, "server is NULL");
    if (srv->fake) return BF_OK;
    std::lock_guard<std::mutex> pl(srv->plan_mu);
    bf_status s;
    {
        std::lock_guard<std::mutex> sl(srv->slot_mu);
        s = bf_set_precoders(srv->plan, W_dev, f_host, n_prec, first_id, srv->prep_st);
    }
    if (s != BF_OK || n_prec == 0) return s;
    cudaEvent_t ev = nullptr;
    if (!srv->prep_pool.empty()) {
        ev = srv->prep_pool.back();
        srv->prep_pool.pop_back();
    } else if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
        return bf_fail(srv->plan, BF_ECUDA, "cudaEventCreate failed");
    }
    if (cudaEventRecord(ev, srv->prep_st) != cudaSuccess) {
        srv->prep_pool.push_back(ev);
        return bf_fail(srv->plan, BF_ECUDA, "cudaEventRecord failed");
    }
    srv->prep_pending.push_back({first_id, first_id + n_prec, ev});
    return BF_OK;
}

extern "C" bf_status bf_submit(bf_server srv, const bf_job *job, uint64_t *ticket) {
    if (!srv || !job || !ticket) return bf_fail(srv ? srv->plan : nullptr, BF_EINVAL, "NULL argument");
    if (job->n_groups < 0 || (job->n_groups && !job->groups)) return bf_fail(srv->plan, BF_EINVAL, "bad groups");
    if (job->prec < BF_FP32 || job->prec >= N_PREC) return bf_fail(srv->plan, BF_EINVAL, "bad precision");
    if (job->n_groups && (!job->S_dev || !job->R_dev || ((uintptr_t)job->S_dev & 15) || ((uintptr_t)job->R_dev & 15)))
        return bf_fail(srv->plan, BF_EINVAL, "S_dev and R_dev must be non-NULL and 16-byte aligned");
    JobRec rec;
    rec.submit_ns = bf_now_ns();
    {
        std::lock_guard<std::mutex> sl(srv->slot_mu);
        const int *f_slot = srv->fake ? nullptr : srv->plan->f_slot.data();
        for (int g = 0; g < job->n_groups; ++g) {
            const bf_group &gr = job->groups[g];
            if (gr.n_blocks < 0 || gr.s_off < 0 || gr.r_off < 0 || (gr.s_off & 15) || (gr.r_off & 15))
                return bf_fail(srv->plan, BF_EINVAL, "group %d: bad block count or offsets", g);
            if (!srv->fake && (gr.prec_id < 0 || gr.prec_id >= srv->plan->cap || f_slot[gr.prec_id] < 0))
                return bf_fail(srv->plan, BF_ENOTFOUND, "group %d: precoder slot %d is not set", g, gr.prec_id);
            bf_group a = gr;
            a.s_off += (int64_t)(uintptr_t)job->S_dev;
            a.r_off += (int64_t)(uintptr_t)job->R_dev;
            rec.groups.push_back(a);
            if (g == 0 || gr.prec_id < rec.slot_lo) rec.slot_lo = gr.prec_id;
            if (g == 0 || gr.prec_id + 1 > rec.slot_hi) rec.slot_hi = gr.prec_id + 1;
        }
        rec.bytes = srv->fake ? 0 : job_bytes(f_slot, job);
        if (srv->fake)
            for (int g = 0; g < job->n_groups; ++g)
                rec.bytes += (int64_t)job->groups[g].n_blocks * (int64_t)R_BLOCK_BYTES;
    }
    rec.cell = job->cell;
    rec.prec = job->prec;
    rec.arrival_ns = job->arrival_ns ? job->arrival_ns : rec.submit_ns;
    std::lock_guard<std::mutex> lk(srv->mu);
    if (rec.bytes > srv->cfg.hbm_budget_bytes) {
        srv->stats.rejected_budget++;
        return bf_fail(srv->plan, BF_EBUDGET, "job needs %lld bytes, budget is %lld", (long long)rec.bytes,
                       (long long)srv->cfg.hbm_budget_bytes);
    }
    if ((int)srv->queue.size() >= srv->cfg.queue_capacity) {
        srv->stats.rejected_full++;
        return bf_fail(srv->plan, BF_EAGAIN, "queue full (%d jobs)", srv->cfg.queue_capacity);
    }
    const uint64_t t = srv->next_ticket++;
    srv->jobs.emplace(t, std::move(rec));
    srv->queue.push_back(t);
    srv->stats.submitted++;
    *ticket = t;
    srv->cv_work.notify_one();
    return BF_OK;
}

static bf_status retire(bf_server srv, std::unordered_map<uint64_t, JobRec>::iterator it, double *latency_us) {
    if (latency_us) *latency_us = (it->second.done_ns - it->second.arrival_ns) * 1e-3;
    const bf_status st = it->second.status;
    srv->jobs.erase(it);
    return st;
}

extern "C" bf_status bf_poll(bf_server srv, uint64_t ticket, int *done, double *latency_us) {
    if (!srv || !done) return bf_fail(srv ? srv->plan : nullptr, BF_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(srv->mu);
    auto it = srv->jobs.find(ticket);
    if (it == srv->jobs.end()) return bf_fail(srv->plan, BF_ENOTFOUND, "unknown ticket %llu", (unsigned long long)ticket);
    *done = it->second.state == DONE;
    if (!*done) return BF_OK;
    return retire(srv, it, latency_us);
}

extern "C" bf_status bf_wait(bf_server srv, uint64_t ticket, int64_t timeout_us, double *latency_us) {
    if (!srv) return bf_fail(nullptr, BF_EINVAL, "server is NULL");
    std::unique_lock<std::mutex> lk(srv->mu);
    auto it = srv->jobs.find(ticket);
    if (it == srv->jobs.end()) return bf_fail(srv->plan, BF_ENOTFOUND, "unknown ticket %llu", (unsigned long long)ticket);
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::microseconds(std::max<int64_t>(0, timeout_us));
    const bool ok = srv->cv_done.wait_until(lk, deadline, [&] {
        auto i = srv->jobs.find(ticket);
        return i != srv->jobs.end() && i->second.state == DONE;
    });
    if (!ok) return bf_fail(srv->plan, BF_ETIMEOUT, "job %llu not done after %lld us", (unsigned long long)ticket,
                            (long long)timeout_us);
    return retire(srv, srv->jobs.find(ticket), latency_us);
}

extern "C" bf_status bf_serve_pause(bf_server srv, int32_t paused) {
    if (!srv) return bf_fail(nullptr, BF_EINVAL, "server is NULL");
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->paused = paused != 0;
    srv->cv_work.notify_all();
    return BF_OK;
}

extern "C" bf_status bf_serve_set_budget(bf_server srv, int64_t hbm_budget_bytes) {
    if (!srv) return bf_fail(nullptr, BF_EINVAL, "server is NULL");
    if (hbm_budget_bytes <= 0) return bf_fail(srv->plan, BF_EINVAL, "budget must be positive");
    std::lock_guard<std::mutex> lk(srv->mu);
    for (uint64_t t : srv->queue) {
        const auto it = srv->jobs.find(t);
        if (it != srv->jobs.end() && it->second.bytes > hbm_budget_bytes)
            return bf_fail(srv->plan, BF_EBUSY, "a queued job needs %lld bytes, more than %lld",
                           (long long)it->second.bytes, (long long)hbm_budget_bytes);
    }
    srv->cfg.hbm_budget_bytes = hbm_budget_bytes;
    srv->cv_work.notify_all();
    return BF_OK;
}

extern "C" bf_status bf_serve_get_stats(bf_server srv, bf_serve_stats *out) {
    if (!srv || !out) return bf_fail(srv ? srv->plan : nullptr, BF_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(srv->mu);
    *out = srv->stats;
    return BF_OK;
}

extern "C" bf_status bf_serve_replay(bf_server srv, const bf_replay_item *items, int32_t n, int64_t start_ns,
                                     uint64_t *tickets, int64_t *late) {
    if (!srv || n < 0 || (n > 0 && (!items || !tickets)))
        return bf_fail(srv ? srv->plan : nullptr, BF_EINVAL, "bad arguments");
    int64_t n_late = 0;
    bf_status s = BF_OK;
    for (int32_t i = 0; i < n && s == BF_OK; ++i) {
        const bf_replay_item &it = items[i];
        bf_job job = it.job;
        job.arrival_ns = start_ns + it.job.arrival_ns;
        while (bf_now_ns() < job.arrival_ns) {
        }
        if (it.W_dev) s = bf_serve_set_precoders(srv, it.W_dev, it.f_host, it.n_prec, it.first_id);
        tickets[i] = 0;
        if (s != BF_OK || (!job.S_dev && job.n_groups == 0)) continue;
        if (bf_now_ns() - job.arrival_ns > 50000) ++n_late;
        s = bf_submit(srv, &job, &tickets[i]);
    }
    if (late) *late = n_late;
    return s;
}
