// sg_serve.cu -- a continuous-batching request loop for sparse diffusion jobs.
//
// Jobs (a shell or band activation, a seed, a step count) are submitted at
// any time.  Everything runs on the server's stream, and each sg_server_tick
// waits once, for the work the previous tick queued:
//   1. the jobs of the previous tick's step advance, and jobs whose step count
//      is reached retire -- their last sum is kept, their grid is destroyed,
//      and submit/admit/done times are recorded (host steady clock);
//   2. the jobs whose admission the previous tick queued join: their counts
//      reached the host behind that step;
//   3. ONE batched fused step (diffuse7 -> box27 -> sum, the batched
//      persistent kernel) is launched over every resident job, so jobs
//      admitted while others are running share the launch;
//   4. while it runs, pending jobs are admitted, first come first served,
//      while a slot is free and the device's free memory (cudaMemGetInfo)
//      covers the job's footprint plus the configured reserve: the host
//      allocates the job's grid and queues its initialisation, activation,
//      list, fill and count behind the step (the step holds every SM, so the
//      device runs them when it ends);
//   5. one event is recorded behind all of it.
// The host's share of admission (bounds, allocation, launches) thus overlaps
// the device's step, and the device runs the admitted jobs' kernels between
// two steps without waiting for the host.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <deque>
#include <new>
#include <unordered_map>
#include <vector>

#include "../../include/sgrid.h"
#include "sg_device.h"

using namespace sg;

namespace {

double now_s()
{
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct Job {
    int64_t id = 0;
    sg_job_desc desc{};
    int state = SG_JOB_PENDING;
    int steps_done = 0;
    int parity = 0;
    long long n_active = 0;
    long long n_leaves = 0;
    double sum = 0.0;
    double t_submit = 0, t_admit = 0, t_done = 0;
    sg_grid *grid = nullptr;
    BatchGrid items[2];
    int cnt_slot = -1;  // its run-record counts in the server's pinned array while joining
};

// Leaves a shell can touch: root cells whose box can meet the band (the same
// bounding test the activation kernel uses) -- an upper bound on the list.
long long shell_leaf_bound(const sg_job_desc &d)
{
    const int L = 8, N = d.res, R = N / L;
    auto range = [&](int c, long long &mn, long long &mx) {
        const long long e0 = 2LL * c * L + 1 - N, e1 = 2LL * (c * L + L - 1) + 1 - N;
        long long lo = (e0 > 0) ? e0 : (e1 < 0 ? -e1 : ((e0 & 1) ? 1 : 0));
        long long hi = std::max(-e0, e1);
        mn = lo * lo;
        mx = hi * hi;
    };
    std::vector<long long> mn(R), mx(R);
    for (int c = 0; c < R; ++c) range(c, mn[c], mx[c]);
    long long count = 0;
    for (int a = 0; a < R; ++a)
        for (int b = 0; b < R; ++b)
            for (int c = 0; c < R; ++c) {
                const long long dmin = mn[a] + mn[b] + mn[c], dmax = mx[a] + mx[b] + mx[c];
                const bool lo_ok = d.lo_strict ? (dmax > d.lo2) : (dmax >= d.lo2);
                if (lo_ok && dmin < d.hi2) ++count;
            }
    return count;
}

size_t job_footprint(const sg_job_desc &d, long long leaves)
{
    const long long R = d.res / 8;
    // 3 fields + mask + nbr + region masks + list, per leaf; root + need per cell
    return size_t(leaves + 1) * (3 * 2048 + 64 + 108 + 160 + 8) + size_t(R * R * R) * 5 + (1 << 20);
}

}  // namespace

struct sg_server {
    sg_server_desc desc{};
    cudaStream_t stream = nullptr;
    cudaEvent_t tick_done = nullptr;  // behind the last tick's step and admissions
    bool in_flight = false;
    std::vector<Job *> in_step;       // the jobs of the in-flight step, in item order
    std::vector<Job *> joining;       // admissions queued behind the in-flight step
    int32_t *host_cnt = nullptr;      // pinned, 3 run-record counts per joining job
    std::deque<Job *> pending;
    std::vector<Job *> resident;
    std::unordered_map<int64_t, Job *> jobs;
    int64_t next_id = 1;
    BatchGrid *dev_items = nullptr;
    double *dev_acc = nullptr;
    BatchGrid *host_items = nullptr;  // pinned
    double *host_acc = nullptr;       // pinned
    void *dev_block = nullptr;
    sg_server_stats stats{};
    int num_sms = 0;
};

namespace {

void *srv_alloc(sg_server *s, size_t bytes)
{
    void *p = nullptr;
    if (s->desc.alloc) return s->desc.alloc(bytes, s->desc.alloc_ctx);
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void srv_free(sg_server *s, void *p)
{
    if (!p) return;
    if (s->desc.free) s->desc.free(p, s->desc.alloc_ctx);
    else cudaFree(p);
}

void retire(sg_server *s, Job *j, int state)
{
    if (j->grid) {
        sg_destroy(j->grid);
        j->grid = nullptr;
    }
    j->state = state;
    j->t_done = now_s();
    if (state == SG_JOB_DONE) s->stats.completed++;
    else s->stats.failed++;
}

// Create a job's grid and queue its activation, list, fill and the copies of
// its counts to the host (pinned slot cnt_slot); returns SG_OK or an error.
int admit(sg_server *s, Job *j, long long leaves)
{
    sg_desc d{};
    d.res = j->desc.res;
    d.leaf_log2 = 3;
    d.n_fields = 3;
    d.max_sums = 1;
    d.max_leaves = std::max(1LL, leaves);
    d.scratch_mask = 0b010;
    d.alloc = s->desc.alloc;
    d.free = s->desc.free;
    d.alloc_ctx = s->desc.alloc_ctx;
    int rc = grid_create(&d, (void *)s->stream, &j->grid, false);
    if (rc) return rc;
    if ((rc = sg_activate_shell(j->grid, j->desc.lo2, j->desc.hi2, j->desc.lo_strict))) return rc;
    if ((rc = sg_list_gen(j->grid))) return rc;
    if ((rc = sg_fill_hash(j->grid, 0, j->desc.seed))) return rc;
    return grid_prepare_batch_async(j->grid, 0, 1, 2, s->host_cnt + 3 * j->cnt_slot);
}

}  // namespace

extern "C" {

int sg_server_create(const sg_server_desc *desc, void *cuda_stream, sg_server **out)
{
    if (!desc || !out || desc->max_jobs < 1 || desc->max_jobs > kMaxBatch || desc->hbm_reserve < 0 ||
        (desc->warps_per_cta != 2 && desc->warps_per_cta != 4 && desc->warps_per_cta != 8) ||
        (desc->alloc == nullptr) != (desc->free == nullptr))
        return SG_ERR_INVALID;
    *out = nullptr;
    sg_server *s = new (std::nothrow) sg_server();
    if (!s) return SG_ERR_OOM;
    s->desc = *desc;
    s->stream = (cudaStream_t)cuda_stream;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&s->num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        delete s;
        return SG_ERR_CUDA;
    }
    const size_t items_bytes = sizeof(BatchGrid) * desc->max_jobs;
    const size_t acc_bytes = sizeof(double) * desc->max_jobs;
    s->dev_block = srv_alloc(s, items_bytes + acc_bytes + 256);
    if (!s->dev_block) {
        delete s;
        return SG_ERR_OOM;
    }
    s->dev_items = (BatchGrid *)s->dev_block;
    s->dev_acc = (double *)((char *)s->dev_block + ((items_bytes + 255) & ~size_t(255)));
    if (cudaMallocHost((void **)&s->host_items, items_bytes) != cudaSuccess ||
        cudaMallocHost((void **)&s->host_acc, acc_bytes) != cudaSuccess) {
        cudaGetLastError();
        if (s->host_items) cudaFreeHost(s->host_items);
        srv_free(s, s->dev_block);
        delete s;
        return SG_ERR_OOM;
    }
    if (cudaMallocHost((void **)&s->host_cnt, sizeof(int32_t) * 3 * desc->max_jobs) != cudaSuccess ||
        cudaEventCreateWithFlags(&s->tick_done, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        if (s->host_cnt) cudaFreeHost(s->host_cnt);
        cudaFreeHost(s->host_items);
        cudaFreeHost(s->host_acc);
        srv_free(s, s->dev_block);
        delete s;
        return SG_ERR_CUDA;
    }
    *out = s;
    return SG_OK;
}

int sg_server_submit(sg_server *s, const sg_job_desc *job, int64_t *job_id)
{
    if (!s || !job || job->res <= 0 || job->res % 8 || job->res > 4096 || job->steps < 1 || job->seed < 0 ||
        job->seed >= (1LL << 24) || job->out_cap < 0)
        return SG_ERR_INVALID;
    Job *j = new (std::nothrow) Job();
    if (!j) return SG_ERR_OOM;
    j->id = s->next_id++;
    j->desc = *job;
    j->t_submit = now_s();
    s->pending.push_back(j);
    s->jobs[j->id] = j;
    s->stats.submitted++;
    if (job_id) *job_id = j->id;
    return SG_OK;
}

int sg_server_tick(sg_server *s)
{
    if (!s) return SG_ERR_INVALID;
    // the work the previous tick queued: its step, then its admissions
    if (s->in_flight || !s->joining.empty())
        if (cudaEventSynchronize(s->tick_done) != cudaSuccess) return SG_ERR_CUDA;
    // 1. the step's jobs advance; those that reached their count retire
    if (s->in_flight) {
        s->in_flight = false;
        for (size_t i = 0; i < s->in_step.size(); ++i) {
            Job *j = s->in_step[i];
            j->steps_done++;
            j->parity ^= 1;
            sg_swap(j->grid, 0, 2);
            j->sum = s->host_acc[i];
            s->stats.voxel_steps += (double)j->n_active;
        }
        s->in_step.clear();
        std::vector<Job *> still;
        still.reserve(s->resident.size());
        for (Job *j : s->resident) {
            if (j->steps_done < j->desc.steps) {
                still.push_back(j);
                continue;
            }
            // the result: field index 0 names the latest x after the swap
            int state = SG_JOB_DONE;
            if (j->desc.out_values) {
                int64_t na = 0;
                if (j->n_active > j->desc.out_cap ||
                    sg_read_field_active(j->grid, 0, j->desc.out_cap, &na, j->desc.out_values) != SG_OK)
                    state = SG_JOB_FAILED;
            }
            retire(s, j, state);
        }
        s->resident.swap(still);
    }
    // 2. the admissions queued behind that step join
    for (Job *j : s->joining) {
        long long na = 0;
        if (grid_prepare_batch_finish(j->grid, 0, 1, 2, s->host_cnt + 3 * j->cnt_slot, j->items, &na) != SG_OK) {
            retire(s, j, SG_JOB_FAILED);
            continue;
        }
        j->n_active = na;
        j->n_leaves = j->items[0].n;
        s->resident.push_back(j);
    }
    s->joining.clear();
    // 3. one batched step over every resident job
    const int n = (int)s->resident.size();
    if (n > 0) {
        int tri = 0;
        for (int i = 0; i < n; ++i) {
            Job *j = s->resident[i];
            s->host_items[i] = j->items[j->parity];
            s->host_items[i].tri0 = tri;
            tri += j->items[0].tasks;
        }
        if (cudaMemcpyAsync(s->dev_items, s->host_items, sizeof(BatchGrid) * n, cudaMemcpyHostToDevice, s->stream) !=
                cudaSuccess ||
            cudaMemsetAsync(s->dev_acc, 0, sizeof(double) * n, s->stream) != cudaSuccess)
            return SG_ERR_CUDA;
        launch_batch_diffuse_box(s->dev_items, n, tri, s->desc.coef, s->dev_acc, s->desc.warps_per_cta, s->num_sms,
                                 s->stream);
        if (cudaPeekAtLastError() != cudaSuccess ||
            cudaMemcpyAsync(s->host_acc, s->dev_acc, sizeof(double) * n, cudaMemcpyDeviceToHost, s->stream) !=
                cudaSuccess)
            return SG_ERR_CUDA;
        s->in_step = s->resident;
        s->in_flight = true;
        s->stats.ticks++;
        s->stats.launches++;
    }
    // 4. admission, while the step runs
    while (!s->pending.empty() && (int)(s->resident.size() + s->joining.size()) < s->desc.max_jobs) {
        Job *j = s->pending.front();
        const long long bound = shell_leaf_bound(j->desc);
        size_t free_b = 0, total_b = 0;
        if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return SG_ERR_CUDA;
        if (free_b < job_footprint(j->desc, bound) + (size_t)s->desc.hbm_reserve) {
            if (s->resident.empty() && s->joining.empty()) {  // can never fit: fail it instead of waiting forever
                s->pending.pop_front();
                retire(s, j, SG_JOB_FAILED);
                continue;
            }
            s->stats.admission_waits++;
            break;
        }
        s->pending.pop_front();
        j->cnt_slot = (int)s->joining.size();
        if (admit(s, j, bound) != SG_OK) {
            retire(s, j, SG_JOB_FAILED);
            continue;
        }
        j->state = SG_JOB_RUNNING;
        j->t_admit = now_s();
        s->joining.push_back(j);
    }
    // 5. one event behind everything queued
    if ((s->in_flight || !s->joining.empty()) && cudaEventRecord(s->tick_done, s->stream) != cudaSuccess)
        return SG_ERR_CUDA;
    return SG_OK;
}

int sg_server_job(sg_server *s, int64_t job_id, sg_job_status *out)
{
    if (!s || !out) return SG_ERR_INVALID;
    auto it = s->jobs.find(job_id);
    if (it == s->jobs.end()) return SG_ERR_INVALID;
    const Job *j = it->second;
    out->state = j->state;
    out->steps_done = j->steps_done;
    out->n_active = j->n_active;
    out->sum = j->sum;
    out->t_submit = j->t_submit;
    out->t_admit = j->t_admit;
    out->t_done = j->t_done;
    return SG_OK;
}

int sg_server_release(sg_server *s, int64_t job_id)
{
    if (!s) return SG_ERR_INVALID;
    auto it = s->jobs.find(job_id);
    if (it == s->jobs.end()) return SG_ERR_INVALID;
    Job *j = it->second;
    // a retired job is in no queue or resident set any more, only in jobs
    if (j->state != SG_JOB_DONE && j->state != SG_JOB_FAILED) return SG_ERR_INVALID;
    s->jobs.erase(it);
    delete j;
    return SG_OK;
}

int sg_server_get_stats(sg_server *s, sg_server_stats *out)
{
    if (!s || !out) return SG_ERR_INVALID;
    *out = s->stats;
    out->resident = (int32_t)(s->resident.size() + s->joining.size());
    out->pending = (int32_t)s->pending.size();
    return SG_OK;
}

int sg_server_destroy(sg_server *s)
{
    if (!s) return SG_OK;
    cudaStreamSynchronize(s->stream);
    for (auto &kv : s->jobs) {
        if (kv.second->grid) sg_destroy(kv.second->grid);
        delete kv.second;
    }
    srv_free(s, s->dev_block);
    if (s->host_items) cudaFreeHost(s->host_items);
    if (s->host_acc) cudaFreeHost(s->host_acc);
    if (s->host_cnt) cudaFreeHost(s->host_cnt);
    cudaEventDestroy(s->tick_done);
    delete s;
    return SG_OK;
}

}  // extern "C"
