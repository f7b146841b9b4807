// Served culling with continuous batching.
//
// Clients submit culling jobs (a set of eyes against a device-resident light hierarchy and
// shift tile) from any thread. A scheduler thread owned by the server:
//   * admits waiting jobs in arrival order while their output reservation fits the HBM
//     budget, giving each a slot of device counters and an output buffer;
//   * runs the GPU as a sequence of slices: each slice is one persistent batched traversal
//     over up to slice_eyes of the admitted jobs' remaining eyes, oldest job first, so a
//     job that arrives while others are on the GPU joins a slice as soon as the older jobs
//     leave room, and its work overlaps theirs;
//   * alternates slices between two streams, so the next slice's blocks fill the SMs as
//     the previous slice drains (no per-slice tail), and keeps at most kRing slices
//     enqueued, so admission reacts within about one slice;
//   * completes a job when the slice holding its last eyes finishes, publishing its pair
//     count and node visits.
// The device never waits on the host: all scheduling happens between launches, so no
// kernel spins on a queue and nothing can hang a GPU. A job's result is independent of
// which other jobs shared its slices (each frame of a slice is traversed exactly as
// hrr_cull would).
#include <chrono>
#include <algorithm>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "hrr_internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;

constexpr int kRing = 2;  // slices enqueued at once (one running, one waiting)
constexpr size_t kSlotWords = 3;  // device counters per job slot: accepted, visits, flags

struct Job {
    uint64_t ticket = 0;
    hrr_job desc{};
    const uint32_t *tile = nullptr;
    uint32_t tile_w = 0, tile_h = 0;
    hrr_tile_buf *ctx_tile = nullptr;  // the submitting context's tile, when the job reads it
    int slot = -1;
    uint2 *pairs = nullptr;
    uint64_t bytes = 0;
    uint32_t next_eye = 0;
    bool admitted = false;
    bool all_launched = false;
    bool done = false;
    cudaEvent_t done_ev = nullptr;
    int status = HRR_PENDING;
    uint64_t count = 0, visits = 0;
    Clock::time_point t_submit, t_admit, t_done;
};

}  // namespace

struct hrr_server {
    int device = 0, sm_count = 0;
    hrr_tuning tuning{};
    cudaStream_t stream = nullptr;              // slice stream 0 (also for frees)
    cudaStream_t slice_stream[kRing] = {};      // slice k runs on slice_stream[k]
    cudaMemPool_t pool = nullptr;               // job outputs; keeps freed memory for reuse
    int last_slice = -1;                        // ring entry of the most recent slice
    uint64_t budget = 0, used = 0;
    uint32_t slice_eyes = 0, max_slots = 0;
    uint32_t slice_min_eyes = 1u << 16;         // a slice may end after a finishing job past this
    unsigned long long *dev_counts = nullptr;   // kSlotWords per slot: accepted, visits, job flags
    unsigned long long *host_counts = nullptr;  // pinned copies
    std::vector<hrr_cull_frame_t> host_frames[kRing];  // slice descriptors (kernel parameters)
    unsigned long long *dev_misc = nullptr;     // 2 per ring entry: cursor, flags
    unsigned grid_max = 1;                      // blocks of a full slice's traversal
    void *spill[kRing] = {};                    // traversal stack spill area per ring entry
    uint32_t spill_height = 0;                  // tallest tree the spill areas are sized for
    unsigned long long *host_flags = nullptr;   // pinned, 1 per ring entry
    cudaEvent_t slice_done[kRing] = {};
    cudaEvent_t setup_done[kRing] = {};          // after a slice's allocations, resets, copies
    bool slice_busy[kRing] = {};
    uint64_t slice_seq[kRing] = {};             // order in which ring entries were filled
    std::vector<Job *> slice_jobs[kRing];
    std::vector<int> free_slots;
    std::deque<Job *> pending;
    std::vector<Job *> active;
    std::map<uint64_t, Job *> jobs;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::thread thread;
    bool stop = false;
    uint64_t next_ticket = 1;
    uint64_t launches = 0, slices = 0, jobs_done = 0;
    uint32_t max_active = 0;
    std::string err;
};

namespace {

double seconds(Clock::duration d) { return std::chrono::duration<double>(d).count(); }

// Finish every job whose last slice has completed, and free finished slice entries.
void reap(hrr_server *s) {
    for (int k = 0; k < kRing; ++k) {
        if (s->slice_busy[k] && cudaEventQuery(s->slice_done[k]) == cudaSuccess) {
            s->slice_busy[k] = false;
            if (s->host_flags[k])
                for (Job *j : s->slice_jobs[k]) j->status = HRR_ERR_DEVICE;
            s->slice_jobs[k].clear();
        }
    }
    for (size_t i = 0; i < s->active.size();) {
        Job *j = s->active[i];
        if (j->all_launched && cudaEventQuery(j->done_ev) == cudaSuccess) {
            const unsigned long long *c = s->host_counts + kSlotWords * (size_t)j->slot;
            j->count = c[0];
            j->visits = c[1];
            if (j->status == HRR_PENDING) {
                if (c[2] & HRR_FLAG_NONFINITE) j->status = HRR_ERR_INVALID_ARG;  // refit lights
                else if (c[2] & HRR_FLAG_TOPOLOGY) j->status = HRR_ERR_DEVICE;
                else j->status = j->count > j->desc.cap ? HRR_ERR_OVERFLOW : HRR_OK;
            }
            j->t_done = Clock::now();
            j->done = true;
            s->free_slots.push_back(j->slot);
            j->slot = -1;
            s->active.erase(s->active.begin() + (long)i);  // keep admission order
            ++s->jobs_done;
            s->cv_done.notify_all();
        } else {
            ++i;
        }
    }
}

void fail_job(hrr_server *s, Job *j, int status) {
    j->status = status;
    j->done = true;
    j->t_done = Clock::now();
    ++s->jobs_done;
    s->cv_done.notify_all();
}

// Admit waiting jobs in arrival order while a slot is free and their output fits.
void admit(hrr_server *s) {
    while (!s->pending.empty() && !s->free_slots.empty()) {
        Job *j = s->pending.front();
        if (j->bytes > s->budget) {  // can never fit
            s->pending.pop_front();
            fail_job(s, j, HRR_ERR_OOM);
            continue;
        }
        if (s->used + j->bytes > s->budget) break;
        s->pending.pop_front();
        s->used += j->bytes;  // the buffer itself is allocated on the job's first slice stream
        j->slot = s->free_slots.back();
        s->free_slots.pop_back();
        j->t_admit = Clock::now();
        j->admitted = true;
        s->active.push_back(j);
        if (s->active.size() > s->max_active) s->max_active = (uint32_t)s->active.size();
    }
}

// Size both ring entries' stack spill areas for trees up to the given height (once per
// taller tree; waits for the slices in flight). False if the memory is not there.
bool ensure_spill(hrr_server *s, uint32_t height) {
    if (height <= s->spill_height && s->spill[0]) return true;
    for (int k = 0; k < kRing; ++k) cudaStreamSynchronize(s->slice_stream[k]);
    const size_t bytes = hrr_cull_spill_entries(s->grid_max, height, s->tuning) * sizeof(uint2);
    for (int k = 0; k < kRing; ++k) {
        if (s->spill[k]) cudaFree(s->spill[k]);
        s->spill[k] = nullptr;
    }
    s->spill_height = 0;
    for (int k = 0; k < kRing; ++k) {
        if (cudaMalloc(&s->spill[k], bytes) != cudaSuccess) {
            cudaGetLastError();
            for (int i = 0; i <= k; ++i) {
                if (s->spill[i]) cudaFree(s->spill[i]);
                s->spill[i] = nullptr;
            }
            return false;
        }
    }
    s->spill_height = height;
    return true;
}

// Enqueue one slice: up to slice_eyes of the admitted jobs' remaining eyes, taken in
// admission order (the oldest job first). Each job thus finishes as early as its place in
// the queue allows, the next jobs' eyes fill the GPU while the older ones drain, and only a
// few hierarchies are live in L2 at a time. Returns false when there was nothing to do.
bool enqueue_slice(hrr_server *s, int k) {
    cudaStream_t st = s->slice_stream[k];
    bool any = false;
    for (Job *j : s->active) any |= !j->all_launched;
    if (!any) return false;
    // A job continuing from the previous slice (other stream) needs that slice's setup
    // (its buffer allocation and counter reset) to have happened first.
    if (s->last_slice >= 0 && s->last_slice != k) cudaStreamWaitEvent(st, s->setup_done[s->last_slice], 0);
    std::vector<Job *> work;
    std::vector<uint32_t> takes;
    uint64_t budget = s->slice_eyes;
    for (Job *j : s->active) {
        if (j->all_launched) continue;
        if (budget == 0 || work.size() == HRR_CULL_MAX_FRAMES) break;
        const bool refit = j->next_eye == 0 && j->desc.refit.x != nullptr;
        if (refit) {
            // The refit changes the tree under every later reader: it starts a slice in
            // which no earlier job reads that tree, after everything in flight.
            bool shared = false;
            for (Job *w : work) shared |= w->desc.tree == j->desc.tree;
            if (shared) break;
            for (int o = 0; o < kRing; ++o)
                if (o != k && s->slice_busy[o]) cudaStreamWaitEvent(st, s->slice_done[o], 0);
        }
        if (j->next_eye == 0) {  // first slice of the job: its buffer and counters
            void *p = nullptr;
            if (j->bytes && cudaMallocFromPoolAsync(&p, j->bytes, s->pool, st) != cudaSuccess) {
                cudaGetLastError();
                j->status = HRR_ERR_OOM;  // completes (with no pairs) like any other job
            }
            j->pairs = static_cast<uint2 *>(p);
            unsigned long long *c = s->dev_counts + kSlotWords * (size_t)j->slot;
            cudaMemsetAsync(c, 0, kSlotWords * sizeof(unsigned long long), st);
        }
        if (refit) {  // moved lights: the step before the traversal, in the job's stream
            void *scratch = nullptr;
            if (cudaMallocFromPoolAsync(&scratch, hrr_refit_scratch_bytes(j->desc.tree->n), s->pool, st) != cudaSuccess) {
                cudaGetLastError();
                j->status = HRR_ERR_OOM;
            } else {
                if (hrr_refit_enqueue(const_cast<hrr_tree *>(j->desc.tree), j->desc.refit, scratch,
                                      s->dev_counts + kSlotWords * (size_t)j->slot + 2, st) == cudaSuccess)
                    s->launches += hrr_refit_launches(j->desc.tree);
                cudaFreeAsync(scratch, st);
            }
        }
        const uint32_t take = (uint32_t)std::min<uint64_t>(budget, j->desc.n_eyes - j->next_eye);
        work.push_back(j);
        takes.push_back(take);
        budget -= take;
        // A job completes when its slice does: once a job's last eyes are in, the slice
        // ends (when it already has enough eyes to fill the GPU), so no job waits for the
        // eyes of jobs behind it. The next slice, on the other stream, takes over as this
        // one drains.
        if (take == j->desc.n_eyes - j->next_eye && s->slice_eyes - budget >= s->slice_min_eyes) break;
    }
    if (work.empty()) return false;
    uint32_t height = 0;
    for (Job *j : work) height = std::max(height, j->desc.tree->height);
    const bool have_spill = ensure_spill(s, height);
    hrr_cull_frame_t *h = s->host_frames[k].data();
    unsigned long long cursor = 0;
    uint32_t n = 0;
    std::vector<Job *> finishing;
    for (size_t w = 0; w < work.size(); ++w) {
        Job *j = work[w];
        const uint32_t take = takes[w];
        hrr_cull_frame_t &d = h[n++];
        d = hrr_cull_frame_t{};
        d.ex = j->desc.eyes.x; d.ey = j->desc.eyes.y; d.ez = j->desc.eyes.z;
        d.px = j->desc.eyes.px; d.py = j->desc.eyes.py;
        d.nodes = hrr_cull_records(j->desc.tree, s->tuning);
        d.perm = j->desc.tree->perm;
        d.tile = j->tile; d.tile_w = j->tile_w; d.tile_h = j->tile_h;
        d.pairs = j->pairs;
        d.cap = j->pairs ? j->desc.cap : 0;  // no buffer (allocation failed): count only
        d.counts = s->dev_counts + kSlotWords * (size_t)j->slot;
        d.eye_visits = nullptr;
        d.n_lights = j->desc.tree->n;
        d.shift_offset = j->desc.shift_offset;
        d.tau = j->desc.tau;
        d.eye_begin = j->next_eye;
        d.cursor_begin = cursor;
        cursor += take;
        j->next_eye += take;
        if (j->next_eye == j->desc.n_eyes) finishing.push_back(j);
    }
    cudaMemsetAsync(s->dev_misc + 2 * k, 0, 2 * sizeof(unsigned long long), st);
    cudaEventRecord(s->setup_done[k], st);
    if (!have_spill) {
        for (Job *j : work) j->status = HRR_ERR_OOM;  // completes with no pairs
    } else if (cursor) {
        const unsigned grid = hrr_cull_grid(s->sm_count, s->tuning, true, cursor);
        if (hrr_cull_batch_enqueue(grid, h, n, cursor, s->dev_misc + 2 * k, s->dev_misc + 2 * k + 1,
                                   s->spill[k], hrr_cull_spill_cap(s->spill_height, s->tuning.node_width), s->tuning,
                                   st) == cudaSuccess)
            ++s->launches;
    }
    cudaMemcpyAsync(&s->host_flags[k], s->dev_misc + 2 * k + 1, sizeof(unsigned long long),
                    cudaMemcpyDeviceToHost, st);
    if (!finishing.empty() && s->last_slice >= 0 && s->last_slice != k)
        // a finishing job may also have eyes in the previous slice, on the other stream:
        // its results are complete only after both
        cudaStreamWaitEvent(st, s->slice_done[s->last_slice], 0);
    for (Job *j : finishing) {
        cudaMemcpyAsync(s->host_counts + kSlotWords * (size_t)j->slot, s->dev_counts + kSlotWords * (size_t)j->slot,
                        kSlotWords * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st);
        cudaEventRecord(j->done_ev, st);
        j->all_launched = true;
    }
    s->slice_jobs[k] = work;
    cudaEventRecord(s->slice_done[k], st);
    s->slice_busy[k] = true;
    s->slice_seq[k] = s->slices;
    s->last_slice = k;
    ++s->slices;
    return true;
}

void run(hrr_server *s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        reap(s);
        admit(s);
        if (s->stop && s->pending.empty() && s->active.empty()) break;
        int k = -1;
        for (int i = 0; i < kRing; ++i)
            if (!s->slice_busy[i]) { k = i; break; }
        bool enqueued = false;
        if (k >= 0) enqueued = enqueue_slice(s, k);
        if (enqueued) continue;
        // Nothing to enqueue now: wait for the oldest busy slice, or for new work.
        int busy = -1;
        for (int i = 0; i < kRing; ++i)
            if (s->slice_busy[i] && (busy < 0 || s->slice_seq[i] < s->slice_seq[busy])) busy = i;
        bool finishing = false;
        for (Job *j : s->active) finishing |= j->all_launched;
        if (busy >= 0 || finishing) {
            cudaEvent_t ev = busy >= 0 ? s->slice_done[busy] : nullptr;
            lk.unlock();
            if (ev) cudaEventSynchronize(ev);
            else std::this_thread::sleep_for(std::chrono::microseconds(100));
            lk.lock();
        } else {
            s->cv_work.wait_for(lk, std::chrono::milliseconds(5));
        }
    }
}

void destroy_resources(hrr_server *s) {
    for (auto &kv : s->jobs) {
        Job *j = kv.second;
        if (j->pairs) cudaFreeAsync(j->pairs, s->stream);
        if (j->done_ev) cudaEventDestroy(j->done_ev);
        hrr_tile_release(j->ctx_tile, s->stream);  // every job is done: nothing reads it any more
        delete j;
    }
    for (int k = 0; k < kRing; ++k)
        if (s->slice_stream[k]) cudaStreamSynchronize(s->slice_stream[k]);
    for (int k = 1; k < kRing; ++k)
        if (s->slice_stream[k]) cudaStreamDestroy(s->slice_stream[k]);
    for (int k = 0; k < kRing; ++k) {
        if (s->spill[k]) cudaFree(s->spill[k]);
        if (s->slice_done[k]) cudaEventDestroy(s->slice_done[k]);
        if (s->setup_done[k]) cudaEventDestroy(s->setup_done[k]);
    }
    if (s->dev_counts) cudaFree(s->dev_counts);
    if (s->host_counts) cudaFreeHost(s->host_counts);
    if (s->dev_misc) cudaFree(s->dev_misc);
    if (s->host_flags) cudaFreeHost(s->host_flags);
    if (s->stream) cudaStreamDestroy(s->stream);
    if (s->pool) cudaMemPoolDestroy(s->pool);
    delete s;
}

void fill_result(const Job *j, hrr_job_result *r) {
    if (!r) return;
    r->status = j->done ? j->status : HRR_PENDING;
    r->count = j->count;
    r->visits = j->visits;
    r->dev_pairs = reinterpret_cast<const uint32_t *>(j->pairs);
    r->queue_s = j->admitted ? seconds(j->t_admit - j->t_submit)
                             : (j->done ? seconds(j->t_done - j->t_submit) : seconds(Clock::now() - j->t_submit));
    r->latency_s = j->done ? seconds(j->t_done - j->t_submit) : seconds(Clock::now() - j->t_submit);
}

}  // namespace

extern "C" {

int hrr_server_create(hrr_ctx *ctx, uint64_t hbm_budget_bytes, uint32_t slice_eyes,
                      uint32_t max_jobs, const hrr_tuning *tuning, hrr_server **out) {
    if (!ctx) return HRR_ERR_INVALID_ARG;
    if (!out) return hrr_fail(ctx, HRR_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (max_jobs == 0 || max_jobs > 65535)
        return hrr_fail(ctx, HRR_ERR_INVALID_ARG, "max_jobs must be in [1, 65535]");
    const hrr_tuning tn = tuning ? *tuning : hrr_tuning{};
    if (!hrr_tuning_valid(tn)) return hrr_fail(ctx, HRR_ERR_INVALID_ARG, "invalid tuning");
    hrr_server *s = new (std::nothrow) hrr_server();
    if (!s) return hrr_fail(ctx, HRR_ERR_OOM, "host allocation of the server");
    s->device = ctx->device;
    s->sm_count = ctx->sm_count;
    s->tuning = hrr_tuning_normalized(tn);
    s->budget = hbm_budget_bytes;
    s->slice_eyes = slice_eyes ? slice_eyes : (1u << 20);
    s->grid_max = hrr_cull_grid(ctx->sm_count, s->tuning, true, s->slice_eyes);
    s->max_slots = max_jobs;
    DeviceGuard g(ctx->device);
    cudaError_t e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
    s->slice_stream[0] = s->stream;
    for (int k = 1; k < kRing && e == cudaSuccess; ++k)
        e = cudaStreamCreateWithFlags(&s->slice_stream[k], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(&s->dev_counts, sizeof(unsigned long long) * kSlotWords * max_jobs);
    if (e == cudaSuccess) e = cudaMallocHost(&s->host_counts, sizeof(unsigned long long) * kSlotWords * max_jobs);
    if (e == cudaSuccess) e = cudaMalloc(&s->dev_misc, sizeof(unsigned long long) * 2 * kRing);
    if (e == cudaSuccess) e = cudaMallocHost(&s->host_flags, sizeof(unsigned long long) * kRing);
    for (int k = 0; k < kRing && e == cudaSuccess; ++k) {
        s->host_frames[k].resize(HRR_CULL_MAX_FRAMES);
        e = cudaEventCreateWithFlags(&s->slice_done[k], cudaEventDisableTiming | cudaEventBlockingSync);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->setup_done[k], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
        destroy_resources(s);
        return hrr_cuda_fail(ctx, e, "server allocation");
    }
    if (e == cudaSuccess) {
        // A pool of its own, holding on to freed job outputs up to the budget: a new job's
        // buffer then reuses mapped memory instead of mapping fresh pages.
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = ctx->device;
        e = cudaMemPoolCreate(&s->pool, &props);
        if (e == cudaSuccess) {
            uint64_t keep = hbm_budget_bytes;
            e = cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &keep);
        }
    }
    if (e != cudaSuccess) {
        destroy_resources(s);
        return hrr_cuda_fail(ctx, e, "server memory pool");
    }
    for (uint32_t i = 0; i < max_jobs; ++i) s->free_slots.push_back((int)(max_jobs - 1 - i));
    try {
        s->thread = std::thread(run, s);
    } catch (...) {
        destroy_resources(s);
        return hrr_fail(ctx, HRR_ERR_OOM, "could not start the scheduler thread");
    }
    *out = s;
    return HRR_OK;
}

int hrr_server_submit(hrr_server *s, hrr_ctx *ctx, const hrr_job *job, uint64_t *ticket) {
    if (!s || !job || !ticket) return HRR_ERR_INVALID_ARG;
    const hrr_job &d = *job;
    if (!d.tree || d.tree->device != s->device || !(d.tau >= 0.0f) || !(d.tau < __builtin_huge_valf()) ||
        (d.n_eyes && (!d.eyes.x || !d.eyes.y || !d.eyes.z || !d.eyes.px || !d.eyes.py)))
        return hrr_fail(ctx, HRR_ERR_INVALID_ARG, "job has a NULL or foreign tree, a bad tau or a NULL eye array");
    if (d.refit.x && (!d.refit.y || !d.refit.z || !d.refit.intensity))
        return hrr_fail(ctx, HRR_ERR_INVALID_ARG, "job refit lights are partly NULL");
    if (!hrr_cull_records(d.tree, s->tuning))
        return hrr_fail(ctx, HRR_ERR_INVALID_ARG, "job tree has no records of the server's node width");
    const uint32_t *tile = d.dev_tile;
    uint32_t tw = d.tile_w, th = d.tile_h;
    hrr_tile_buf *ctx_tile = nullptr;
    if (!tile) {
        if (!ctx || !ctx->tile) return hrr_fail(ctx, HRR_ERR_NO_TILE, "job has no tile and no context tile is set");
        tile = hrr_tile_layer(ctx->tile, ctx->tile_w, ctx->tile_h, ctx->tile_d, d.sample_index);
        tw = ctx->tile_w; th = ctx->tile_h;
        ctx_tile = ctx->tile_buf;
    } else if (tw == 0 || th == 0 || tw > 65536 || th > 65536 || d.tile_d > 65536) {
        return hrr_fail(ctx, HRR_ERR_INVALID_ARG, "job tile size is invalid");
    } else {
        tile = hrr_tile_layer(tile, tw, th, d.tile_d, d.sample_index);
    }
    Job *j = new (std::nothrow) Job();
    if (!j) return hrr_fail(ctx, HRR_ERR_OOM, "host allocation of a job");
    j->desc = d;
    j->tile = tile; j->tile_w = tw; j->tile_h = th;
    j->ctx_tile = ctx_tile;
    hrr_tile_retain(ctx_tile);  // released with the job, so a new context tile cannot free it
    j->bytes = d.cap * sizeof(uint2);
    j->t_submit = Clock::now();
    {
        DeviceGuard g(s->device);
        if (cudaEventCreateWithFlags(&j->done_ev, cudaEventDisableTiming) != cudaSuccess) {
            delete j;
            return hrr_fail(ctx, HRR_ERR_CUDA, "event creation");
        }
    }
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) {
        cudaEventDestroy(j->done_ev);
        hrr_tile_release(j->ctx_tile, s->stream);
        delete j;
        return hrr_fail(ctx, HRR_ERR_INVALID_ARG, "server is shutting down");
    }
    j->ticket = s->next_ticket++;
    s->jobs[j->ticket] = j;
    if (d.n_eyes == 0) {
        j->all_launched = true;  // nothing to traverse: completes at once
        j->status = HRR_OK;
        j->done = true;
        j->admitted = true;
        j->t_admit = j->t_done = j->t_submit;
        ++s->jobs_done;
    } else {
        s->pending.push_back(j);
    }
    *ticket = j->ticket;
    s->cv_work.notify_one();
    return HRR_OK;
}

int hrr_server_poll(hrr_server *s, uint64_t ticket, hrr_job_result *res) {
    if (!s) return HRR_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->jobs.find(ticket);
    if (it == s->jobs.end()) return HRR_ERR_INVALID_ARG;
    fill_result(it->second, res);
    return it->second->done ? HRR_OK : HRR_PENDING;
}

int hrr_server_wait(hrr_server *s, uint64_t ticket, double timeout_s, hrr_job_result *res) {
    if (!s) return HRR_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->jobs.find(ticket);
    if (it == s->jobs.end()) return HRR_ERR_INVALID_ARG;
    Job *j = it->second;
    const auto deadline = Clock::now() + std::chrono::duration_cast<Clock::duration>(
                                             std::chrono::duration<double>(timeout_s > 0 ? timeout_s : 0.0));
    while (!j->done) {
        if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && !j->done) {
            fill_result(j, res);
            return HRR_ERR_TIMEOUT;
        }
    }
    fill_result(j, res);
    return HRR_OK;
}

int hrr_server_release(hrr_server *s, uint64_t ticket) {
    if (!s) return HRR_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->jobs.find(ticket);
    if (it == s->jobs.end() || !it->second->done) return HRR_ERR_INVALID_ARG;
    Job *j = it->second;
    DeviceGuard g(s->device);
    if (j->pairs) cudaFreeAsync(j->pairs, s->stream);
    if (j->admitted) s->used -= j->bytes;
    if (j->done_ev) cudaEventDestroy(j->done_ev);
    hrr_tile_release(j->ctx_tile, s->stream);  // the job is done: its slices no longer read the tile
    s->jobs.erase(it);
    delete j;
    s->cv_work.notify_one();
    return HRR_OK;
}

int hrr_server_copy_pairs(hrr_server *s, uint64_t ticket, uint32_t *host_pairs, uint64_t max_pairs,
                          uint64_t *copied) {
    if (!s || (!host_pairs && max_pairs)) return HRR_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->jobs.find(ticket);
    if (it == s->jobs.end() || !it->second->done) return HRR_ERR_INVALID_ARG;
    const Job *j = it->second;
    const uint64_t n = std::min(std::min(j->count, j->desc.cap), max_pairs);
    if (copied) *copied = 0;
    if (n && j->pairs) {
        // The job is done, so its pairs are final; copy them without waiting for the slices
        // still running on the server stream (the caller must not release this ticket
        // concurrently).
        const void *src = j->pairs;
        lk.unlock();
        DeviceGuard g(s->device);
        if (cudaMemcpy(host_pairs, src, n * sizeof(uint2), cudaMemcpyDeviceToHost) != cudaSuccess) return HRR_ERR_CUDA;
    }
    if (copied) *copied = n;
    return HRR_OK;
}

int hrr_server_stats(hrr_server *s, hrr_server_info *info) {
    if (!s || !info) return HRR_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    info->slices = s->slices;
    info->launches = s->launches;
    info->jobs_done = s->jobs_done;
    info->jobs_waiting = s->pending.size();
    info->jobs_active = s->active.size();
    info->max_active = s->max_active;
    info->bytes_reserved = s->used;
    return HRR_OK;
}

int hrr_server_destroy(hrr_server *s) {
    if (!s) return HRR_ERR_INVALID_ARG;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        s->cv_work.notify_one();
    }
    if (s->thread.joinable()) s->thread.join();
    DeviceGuard g(s->device);
    destroy_resources(s);
    return HRR_OK;
}

}  // extern "C"
