/*
 * bf_serve.h -- continuous-batching serving loop around the batched product
 * of bf.h (R = W x S per block, Sec. III).
 *
 * The base station of the paper runs one pipeline instance per CPU core in
 * "continuous mode" over many streams (Sec. II; Sec. III on multi-stream
 * turbo decoding). Here the streams are cells that each emit one beamforming
 * job per transmission time interval (TTI). A server owns one dispatcher
 * thread that
 *   - takes submitted jobs in FIFO order,
 *   - admits a job when a launch slot is free and the bytes of all admitted,
 *     unfinished jobs stay within the HBM budget,
 *   - merges the admitted jobs of one precision (up to max_batch_jobs) into a
 *     single persistent launch on the slot's stream, so jobs that arrive while
 *     others run start at once on another slot and overlap them on the device,
 *   - detects completion by polling the slot's event, stamps each job's
 *     completion time and releases its budget.
 * Results do not depend on what a job is batched with: every element's
 * reduction order is fixed by the precision and f alone.
 *
 * Buffers: the caller keeps S and R of each job resident on the device and
 * owns them; they must stay valid until the job is done. Precoder slots are
 * set through bf_serve_set_precoders so that later launches that read those
 * slots are ordered after the conversion (launches reading other slots are
 * not held back). While a server exists, only the server may use its plan.
 */
#ifndef BF_SERVE_H
#define BF_SERVE_H

#include "bf.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bf_server_s *bf_server;

typedef struct {
    int32_t n_slots;           /* launches in flight at once (1..8), one stream each       */
    int32_t max_batch_jobs;    /* jobs merged into one launch (>= 1)                       */
    int32_t queue_capacity;    /* submitted but not admitted jobs; BF_EAGAIN beyond        */
    int32_t fake_device_us;    /* 0: real GPU. > 0: no CUDA at all; every launch "runs"
                                  for this many microseconds on a host timer (tests of the
                                  admission, batching and failure paths on machines
                                  without a GPU); the plan argument may then be NULL      */
    int64_t hbm_budget_bytes;  /* admission budget (> 0)                                   */
    int32_t deadline_us;       /* per-job latency deadline for the statistics (>= 0; 0: the
                                  0.5 ms TTI of Sec. II's slot timing, 500 us)              */
    int32_t slot_timeout_us;   /* watchdog (>= 0; 0: 50,000 us): a launch whose completion is
                                  not seen this long after it was enqueued fails its jobs
                                  with BF_ETIMEOUT (see bf_poll); its slot and the jobs'
                                  budget stay held until the launch does complete, since the
                                  device may still be writing their R                      */
} bf_serve_config;

typedef struct {
    int32_t cell;              /* submitting cell (statistics only)                        */
    int32_t n_groups;
    const bf_group *groups;    /* host array, copied by bf_submit; offsets relative to
                                  S_dev / R_dev                                            */
    bf_precision prec;         /* complex64 S for every precision (no held S here)         */
    int32_t pad;
    const void *S_dev;
    void *R_dev;
    int64_t arrival_ns;        /* scheduled arrival on the bf_now_ns clock (0 = now);
                                  latency is measured from it                              */
} bf_job;

typedef struct {
    int64_t submitted, completed, launches, rejected_budget, rejected_full;
    int64_t budget_waits;      /* admissions delayed because the budget was full           */
    int64_t max_inflight_bytes;
    int32_t max_busy_slots;    /* most launches seen in flight together                    */
    int32_t max_jobs_per_launch;
    int64_t over_deadline;     /* jobs completed (or timed out) later than the deadline     */
    int64_t timed_out;         /* jobs failed by the watchdog with BF_ETIMEOUT               */
    int64_t deadline_ns, slot_timeout_ns;  /* the limits in use                            */
    /* The job with the largest latency so far, and where its time went:
     * submit = arrival -> bf_submit called (a late caller), queue = bf_submit ->
     * admitted by the dispatcher (budget, free slot, FIFO), launch = admitted ->
     * launch enqueued (host side: waits on precoder conversions, scheduling,
     * the launch call), device = enqueued -> completion seen by the dispatcher. */
    int64_t worst_latency_ns, worst_submit_ns, worst_queue_ns, worst_launch_ns, worst_device_ns;
    /* Over-deadline jobs by the largest of those four parts of their latency. */
    int64_t over_by_submit, over_by_queue, over_by_launch, over_by_device;
    /* The four parts summed over every job that left the engine (divide by
     * completed for the means). */
    int64_t sum_submit_ns, sum_queue_ns, sum_launch_ns, sum_device_ns;
} bf_serve_stats;

/* Monotonic clock (CLOCK_MONOTONIC) in nanoseconds, the clock of arrival_ns. */
int64_t bf_now_ns(void);

/* Start a server on `plan` (NULL with fake_device_us > 0). BF_EINVAL for a bad
 * config; BF_ECUDA when streams or events cannot be created. */
bf_status bf_serve_create(bf_plan plan, const bf_serve_config *cfg, bf_server *out);

/* Stop the dispatcher. Waits up to `timeout_us` for queued and in-flight jobs
 * to finish; returns BF_EBUSY (and keeps the server) if they do not. */
bf_status bf_serve_destroy(bf_server srv, int64_t timeout_us);

/* Set precoder slots like bf_set_precoders; launches admitted after this call
 * returns whose jobs read any of these slots are ordered after the
 * conversion. Consecutive calls do not wait for each other's conversions. */
bf_status bf_serve_set_precoders(bf_server srv, const void *W_dev, const int32_t *f_host,
                                 int32_t n_prec, int32_t first_id);

/* Queue a job; *ticket identifies it. BF_EBUDGET if the job alone exceeds the
 * whole budget, BF_EAGAIN if the queue is full, BF_ENOTFOUND for an unset
 * precoder slot, BF_EINVAL for bad arguments. Never blocks on the GPU. */
bf_status bf_submit(bf_server srv, const bf_job *job, uint64_t *ticket);

/* Non-blocking completion check. *done = 1 when the job has finished; then
 * *latency_us (if not NULL) is completion minus arrival, and the ticket is
 * retired (a later poll gives BF_ENOTFOUND). The return value is then the
 * job's own status: BF_OK, BF_ECUDA for a failed launch, or BF_ETIMEOUT when
 * the watchdog gave its launch up (slot_timeout_us; its R must not be used).
 * BF_ENOTFOUND for unknown tickets. */
bf_status bf_poll(bf_server srv, uint64_t ticket, int *done, double *latency_us);

/* Block until the job is done or `timeout_us` passes (BF_ETIMEOUT; the job
 * stays queued or running and its ticket stays valid). Once the job is done it
 * retires the ticket and returns the job's status like bf_poll (BF_ETIMEOUT
 * there means the watchdog gave the launch up; the ticket is then retired). */
bf_status bf_wait(bf_server srv, uint64_t ticket, int64_t timeout_us, double *latency_us);

/* Hold (1) or resume (0) admission of queued jobs; jobs in flight continue.
 * Used to model a stalled producer. */
bf_status bf_serve_pause(bf_server srv, int32_t paused);

/* Change the HBM admission budget (> 0, BF_EINVAL otherwise). Jobs in flight
 * keep running; later admissions use the new budget, and a larger budget
 * admits waiting jobs at once. BF_EBUSY (budget unchanged) if a queued job
 * needs more than the new budget, since it could then never be admitted. */
bf_status bf_serve_set_budget(bf_server srv, int64_t hbm_budget_bytes);

bf_status bf_serve_get_stats(bf_server srv, bf_serve_stats *out);

/* One entry of an arrival schedule replayed by bf_serve_replay. */
typedef struct {
    bf_job job;                /* arrival_ns relative to the replay's start_ns; S_dev NULL
                                  and n_groups 0: no job (a precoder update only)           */
    const void *W_dev;         /* not NULL: bf_serve_set_precoders(srv, W_dev, f_host,     */
    const int32_t *f_host;     /*   n_prec, first_id) at the item's time, before its job   */
    int32_t n_prec;
    int32_t first_id;
} bf_replay_item;

/* Load generator in native code (the cells of Sec. II's continuous mode, each
 * emitting one job per TTI): on the calling thread, takes the items in order,
 * waits (spinning on bf_now_ns) until start_ns + job.arrival_ns, sets the
 * item's precoders if it carries any, then submits its job with that arrival
 * time (latency counts from it); tickets[i] receives item i's ticket (0 for an
 * update-only item). Items whose time has passed run at once. *late (may be
 * NULL) receives the number of jobs submitted more than 50 us after their
 * arrival. Stops at the first failing call and returns its status; the
 * tickets of the items before it stay valid. BF_EINVAL for bad arguments. */
bf_status bf_serve_replay(bf_server srv, const bf_replay_item *items, int32_t n, int64_t start_ns,
                          uint64_t *tickets, int64_t *late);

#ifdef __cplusplus
}
#endif
#endif /* BF_SERVE_H */
