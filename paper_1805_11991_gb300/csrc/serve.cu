// serve.cu -- request loop with continuous batching.
//
// A server thread owns a CUDA stream and runs the device in steps.  Each step
// is one launch of the persistent count kernel over a slice of every active
// request (an equal share of point evaluations each, about kStepMs of device
// time in all at the rate measured on earlier steps), so requests of very
// different sizes progress together and a request that arrives while others
// run joins at the next step boundary once a slot and enough device memory
// are free.  Field
// tables stay resident in the process-wide table cache.  Each request owns its
// histogram hash; slices of one request add into it across steps, and when
// its last slice is done the hash is compacted and copied out.  Results do not
// depend on how requests were mixed: every slice adds exact integer counts.
#include "hwc_internal.cuh"

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <set>
#include <thread>
#include <tuple>

using namespace hwc;
using Clock = std::chrono::steady_clock;

namespace {

struct Request {
    uint64_t ticket = 0;
    hwc_job_t job{};
    KJob kj{};
    uint64_t next_tile = 0;
    std::vector<void *> allocs;
    uint64_t bytes = 0;
    int state = 0;   // 0 queued, 1 active, 2 done
    int rc = HWC_OK;
    std::string err;
    hwc_hist *result = nullptr;
    bool collected = false;
    Clock::time_point t_submit, t_admit, t_done;
};

}  // namespace

struct hwc_server {
    hwc_server_config_t cfg{};
    int device = 0;
    cudaStream_t stream = nullptr;
    std::thread th;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request *> pending;
    std::vector<Request *> active;
    std::map<uint64_t, Request *> all;
    uint64_t next_ticket = 1;
    bool stop = false;
    uint64_t used_bytes = 0;
    std::set<std::pair<uint32_t, uint32_t>> tables_seen;
    KJob *d_jobs = nullptr;
    uint64_t *d_item_start = nullptr;     // [2 * max_active]
    unsigned long long *d_counters = nullptr;   // [max_active]
    KJob *h_jobs = nullptr;          // pinned staging
    uint64_t *h_item_start = nullptr;
    std::map<std::pair<int, uint32_t>, LaunchShape> shapes;
    unsigned long long *d_wkeys = nullptr;   // two-level kernel: member keys per resident warp
    uint64_t wkeys_slots = 0;
    uint64_t steps = 0;
    double evals_per_ms = 0;   // device rate of earlier steps (running mean); 0 before the first
};

namespace {

// device time a step aims at, and the rate assumed before one was measured
constexpr double kStepMs = 4.0;
constexpr double kFirstEvalsPerMs = 1e9;

// nominal point evaluations of one tile of a job: members per tile (q^2
// for the two-level fan-out, q for the c_0 fan-out, 32 per member tile)
// times sum_k q^k
double tile_evals(const KJob &kj)
{
    const double members = kj.method == 2 ? (double)kj.q * kj.q : (kj.method == 1 ? (double)kj.q : (double)kTileMembers);
    double pts = 0;
    for (uint32_t k = 0; k < kj.g; ++k) pts += kj.Q[k];
    return members * pts;
}

void free_request_device(Request *r)
{
    for (void *p : r->allocs) cudaFree(p);
    r->allocs.clear();
}

template <class T>
int ralloc(Request *r, T **p, uint64_t n)
{
    void *v = nullptr;
    if (cudaMalloc(&v, std::max<uint64_t>(n, 1) * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        return set_error(HWC_ERR_NOMEM, "cudaMalloc failed");
    }
    r->allocs.push_back(v);
    *p = (T *)v;
    return HWC_OK;
}

int shape_for(hwc_server *s, int D, uint32_t method, uint32_t words, uint32_t smem, LaunchShape *out)
{
    auto key = std::make_pair(D * 16 + (int)(method * 4 + words), smem);
    auto it = s->shapes.find(key);
    if (it != s->shapes.end()) {
        *out = it->second;
        return HWC_OK;
    }
    int rc = choose_shape(D, method, words, smem, true, out);
    if (rc) return rc;
    s->shapes[key] = *out;
    return HWC_OK;
}

// admission: allocate the request's hash and clear it (server thread)
int admit(hwc_server *s, Request *r)
{
    KJob &kj = r->kj;
    const uint32_t cap = kj.hmask + 1;
    int rc;
    if ((rc = ralloc(r, &kj.hkeys, cap)) || (rc = ralloc(r, &kj.hcounts, cap)) ||
        (rc = ralloc(r, &kj.stats, 4)) || (rc = ralloc(r, &kj.out_keys, cap)) ||
        (rc = ralloc(r, &kj.out_counts, cap)) || (rc = ralloc(r, &kj.n_out, 1)))
        return rc;
    KJob *d_one = nullptr;
    if ((rc = ralloc(r, &d_one, 1))) return rc;
    HWC_CUDA_TRY(cudaMemcpyAsync(d_one, &kj, sizeof kj, cudaMemcpyHostToDevice, s->stream));
    rc = launch_clear(d_one, 1, nullptr, 0, s->stream);
    if (rc) return rc;
    HWC_CUDA_TRY(cudaStreamSynchronize(s->stream));
    return HWC_OK;
}

// finished request: compact its hash and build the host histogram
int finish(hwc_server *s, Request *r)
{
    KJob *d_one = (KJob *)r->allocs.back();
    int rc = launch_compact(d_one, 1, s->stream);
    if (rc) return rc;
    unsigned long long st[3] = {}, n_out = 0;
    HWC_CUDA_TRY(cudaMemcpyAsync(st, r->kj.stats, sizeof st, cudaMemcpyDeviceToHost, s->stream));
    HWC_CUDA_TRY(cudaMemcpyAsync(&n_out, r->kj.n_out, sizeof n_out, cudaMemcpyDeviceToHost, s->stream));
    HWC_CUDA_TRY(cudaStreamSynchronize(s->stream));
    if (st[2]) return set_error(HWC_ERR_TOO_LARGE, "histogram hash overflowed");
    std::vector<unsigned long long> keys(n_out), cnt(n_out);
    if (n_out) {
        HWC_CUDA_TRY(cudaMemcpy(keys.data(), r->kj.out_keys, n_out * 8, cudaMemcpyDeviceToHost));
        HWC_CUDA_TRY(cudaMemcpy(cnt.data(), r->kj.out_counts, n_out * 8, cudaMemcpyDeviceToHost));
    }
    r->result = hist_from_keys(r->kj, keys.data(), cnt.data(), n_out, st[0]);
    return HWC_OK;
}

void complete(hwc_server *s, Request *r, int rc)
{
    // called with s->mu held
    r->rc = rc;
    if (rc) r->err = hwc_last_error();
    r->state = 2;
    r->t_done = Clock::now();
    free_request_device(r);
    s->used_bytes -= std::min(s->used_bytes, r->bytes);
    s->cv_done.notify_all();
}

void server_loop(hwc_server *s)
{
    cudaSetDevice(s->device);
    const uint32_t max_active = std::max<uint32_t>(1, s->cfg.max_active);
    for (;;) {
        std::vector<Request *> step;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            for (;;) {
                // admit while a slot and memory are free
                while (!s->pending.empty() && s->active.size() < max_active) {
                    Request *r = s->pending.front();
                    if (r->bytes > s->cfg.device_bytes) {
                        s->pending.pop_front();
                        set_error(HWC_ERR_BUSY, "request needs %llu bytes, budget %llu",
                                  (unsigned long long)r->bytes, (unsigned long long)s->cfg.device_bytes);
                        s->used_bytes += r->bytes;
                        complete(s, r, HWC_ERR_BUSY);
                        continue;
                    }
                    if (s->used_bytes + r->bytes > s->cfg.device_bytes) break;
                    s->pending.pop_front();
                    s->used_bytes += r->bytes;
                    lk.unlock();
                    int rc = admit(s, r);
                    lk.lock();
                    if (rc) {
                        complete(s, r, rc);
                        continue;
                    }
                    r->state = 1;
                    r->t_admit = Clock::now();
                    s->active.push_back(r);
                }
                if (!s->active.empty()) break;
                if (s->stop && s->pending.empty()) return;
                s->cv_work.wait(lk);
            }
            step = s->active;
        }

        // one device step: a fair share of tiles of every active request; requests
        // of one degree share a persistent launch
        auto skey = [](const Request *x) { return std::make_tuple(x->kj.d, x->kj.method, x->kj.words); };
        std::stable_sort(step.begin(), step.end(),
                         [&](const Request *x, const Request *y) { return skey(x) < skey(y); });
        const uint32_t n = (uint32_t)step.size();
        std::vector<uint64_t> took(n, 0);
        // equal point evaluations per request, the step about kStepMs in all
        const double req_evals = (s->evals_per_ms > 0 ? s->evals_per_ms : kFirstEvalsPerMs) * kStepMs / n;
        int rc = HWC_OK;
        uint32_t item_off = 0, ngroups = 0;
        struct StepGroup {
            int D;
            uint32_t method, words;
            uint32_t first, n, off;
            uint64_t items;
            uint32_t smem;
            LaunchShape sh;
        };
        std::vector<StepGroup> groups;
        for (uint32_t i = 0; i < n && rc == HWC_OK;) {
            uint32_t e = i;
            uint32_t smem = 0;
            while (e < n && skey(step[e]) == skey(step[i])) smem = std::max(smem, step[e++]->kj.smem_bytes);
            StepGroup G{(int)step[i]->kj.d, step[i]->kj.method, step[i]->kj.words, i, e - i, item_off, 0, smem,
                        LaunchShape()};
            if (G.method == 2) {
                std::vector<Fan2Need> needs;
                for (uint32_t r = i; r < e; ++r) needs.push_back({step[r]->kj.warp_off, step[r]->kj.warp_bytes});
                rc = choose_shape_fan2(G.D, needs.data(), needs.size(), &G.sh, &G.smem);
                if (rc == HWC_OK &&
                    (uint64_t)G.sh.grid * (G.sh.block / 32) * 961ull > s->wkeys_slots)
                    rc = set_error(HWC_ERR_TOO_LARGE, "server key scratch too small");
            } else {
                rc = shape_for(s, G.D, G.method, G.words, smem, &G.sh);
            }
            if (rc) break;
            // per request: its share of the step's point evaluations (req_evals),
            // and at least its share of about 8 work items per CTA of the launch
            // (the tail of a launch then weighs little); with step_items set by
            // the caller, exactly its share of step_items items per launch
            uint64_t budget = s->cfg.step_items ? s->cfg.step_items : (uint64_t)G.sh.grid * 8;
            budget *= (uint64_t)G.sh.item_tiles;
            const uint64_t share = std::max<uint64_t>(G.sh.item_tiles, budget / (e - i));
            uint64_t items = 0;
            for (uint32_t r = i; r < e; ++r) {
                Request *q = step[r];
                KJob sl = q->kj;
                const uint64_t left = q->kj.n_tiles - q->next_tile;
                uint64_t want = share;
                if (!s->cfg.step_items)
                    want = std::max<uint64_t>(want, (uint64_t)(req_evals / tile_evals(q->kj)) + 1);
                const uint64_t t = std::min(left, want);
                took[r] = t;
                if (q->kj.method != 0) {
                    // fan-out tiles are groups; the member range stays the request's
                    sl.first_group = q->kj.first_group + q->next_tile;
                } else {
                    sl.first = q->kj.first + q->next_tile * kTileMembers;
                    sl.count = std::min<uint64_t>(q->kj.count - q->next_tile * kTileMembers, t * kTileMembers);
                }
                sl.n_tiles = t;
                sl.wkeys = s->d_wkeys;
                sl.wkeys_stride = 961;   // q <= 31
                s->h_jobs[r] = sl;
                s->h_item_start[item_off + (r - i)] = items;
                items += (t + G.sh.item_tiles - 1) / G.sh.item_tiles;
            }
            s->h_item_start[item_off + (e - i)] = items;
            G.items = items;
            item_off += (e - i) + 1;
            groups.push_back(G);
            ++ngroups;
            i = e;
        }
        cudaError_t ce = cudaSuccess;
        const Clock::time_point t_step = Clock::now();
        if (rc == HWC_OK) {
            ce = cudaMemcpyAsync(s->d_jobs, s->h_jobs, n * sizeof(KJob), cudaMemcpyHostToDevice, s->stream);
            if (ce == cudaSuccess)
                ce = cudaMemcpyAsync(s->d_item_start, s->h_item_start, item_off * sizeof(uint64_t),
                                     cudaMemcpyHostToDevice, s->stream);
            if (ce == cudaSuccess)
                ce = cudaMemsetAsync(s->d_counters, 0, ngroups * sizeof(unsigned long long), s->stream);
            if (ce != cudaSuccess) rc = set_error(HWC_ERR_CUDA, "step setup: %s", cudaGetErrorString(ce));
        }
        for (size_t g = 0; rc == HWC_OK && g < groups.size(); ++g) {
            const StepGroup &G = groups[g];
            rc = launch_persistent(G.D, G.method, G.words, s->d_jobs + G.first, s->d_item_start + G.off, G.n,
                                   G.items, s->d_counters + g, G.smem, G.sh, s->stream);
        }
        if (rc == HWC_OK) {
            ce = cudaStreamSynchronize(s->stream);
            if (ce != cudaSuccess) rc = set_error(HWC_ERR_CUDA, "step: %s", cudaGetErrorString(ce));
        }
        if (rc == HWC_OK) {   // the step's rate updates the running mean
            const double ms = std::chrono::duration<double, std::milli>(Clock::now() - t_step).count();
            double ev = 0;
            for (uint32_t i = 0; i < n; ++i) ev += (double)took[i] * tile_evals(step[i]->kj);
            if (ms > 0 && ev > 0)
                s->evals_per_ms = s->evals_per_ms > 0 ? 0.5 * s->evals_per_ms + 0.5 * (ev / ms) : ev / ms;
        }
        ++s->steps;

        std::lock_guard<std::mutex> lk(s->mu);
        std::vector<Request *> still;
        for (uint32_t i = 0; i < n; ++i) {
            Request *r = step[i];
            if (rc) {
                complete(s, r, rc);
                continue;
            }
            r->next_tile += took[i];
            if (r->next_tile >= r->kj.n_tiles) {
                int frc = finish(s, r);
                complete(s, r, frc);
            } else {
                still.push_back(r);
            }
        }
        s->active.swap(still);
    }
}

}  // namespace

extern "C" int hwc_serve_open(const hwc_server_config_t *cfg, hwc_server_t **out)
{
    if (!out) return set_error(HWC_ERR_ARG, "out is NULL");
    *out = nullptr;
    int rc = prepare_count_kernels();
    if (rc) return rc;
    hwc_server *s = new hwc_server();
    if (cfg) s->cfg = *cfg;
    if (!s->cfg.device_bytes) s->cfg.device_bytes = 8ull << 30;
    if (!s->cfg.max_active) s->cfg.max_active = 64;
    cudaGetDevice(&s->device);
    const uint32_t m = s->cfg.max_active;
    bool ok = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) == cudaSuccess &&
              cudaMalloc(&s->d_jobs, m * sizeof(KJob)) == cudaSuccess &&
              cudaMalloc(&s->d_item_start, 2 * (m + 1) * sizeof(uint64_t)) == cudaSuccess &&
              cudaMalloc(&s->d_counters, m * sizeof(unsigned long long)) == cudaSuccess &&
              cudaMallocHost(&s->h_jobs, m * sizeof(KJob)) == cudaSuccess &&
              cudaMallocHost(&s->h_item_start, 2 * (m + 1) * sizeof(uint64_t)) == cudaSuccess;
    // every resident warp of the GPU (at most 64 per SM) may hold q^2 <= 961 keys
    s->wkeys_slots = (uint64_t)device_sm_count() * 64 * 961;
    ok = ok && cudaMalloc(&s->d_wkeys, s->wkeys_slots * sizeof(unsigned long long)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        hwc_serve_close(s);
        return set_error(HWC_ERR_NOMEM, "server allocation failed");
    }
    s->th = std::thread(server_loop, s);
    *out = s;
    return HWC_OK;
}

extern "C" int hwc_serve_submit(hwc_server_t *s, const hwc_job_t *job, uint64_t *ticket)
{
    if (!s || !job || !ticket) return set_error(HWC_ERR_ARG, "null argument");
    Request *r = new Request();
    r->job = *job;
    uint64_t fam_n = 0;
    TuneChoice tc;   // a choice the autotuner already made for this class (no measuring here)
    tune_lookup(*job, 0, &tc);
    int rc = fill_kjob(*job, r->kj, &fam_n, 0, &tc);   // validates, builds tables
    if (rc) {
        delete r;
        return rc;
    }
    r->kj.hmask = hash_capacity(r->kj.g, r->kj.q, job->count, 1) - 1;
    r->bytes = 32ull * (r->kj.hmask + 1ull) + 4096;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        for (uint32_t k = 1; k <= job->g; ++k)
            if (s->tables_seen.insert({job->q, k}).second) {
                uint64_t Q = r->kj.Q[k - 1];
                s->used_bytes += 4ull * (Q + 2 * Q + 2 * Q + job->q);   // resident tables
            }
        r->ticket = s->next_ticket++;
        r->t_submit = Clock::now();
        s->all[r->ticket] = r;
        s->pending.push_back(r);
        *ticket = r->ticket;
    }
    s->cv_work.notify_one();
    return HWC_OK;
}

extern "C" int hwc_serve_poll(hwc_server_t *s, uint64_t ticket, uint32_t timeout_ms, hwc_hist_t **out)
{
    if (!s || !out) return set_error(HWC_ERR_ARG, "null argument");
    *out = nullptr;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) return set_error(HWC_ERR_ARG, "unknown ticket %llu", (unsigned long long)ticket);
    Request *r = it->second;
    if (r->state != 2 && timeout_ms > 0)
        s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] { return r->state == 2; });
    if (r->state != 2) return set_error(HWC_ERR_STATE, "request %llu not finished", (unsigned long long)ticket);
    if (r->rc) return set_error(r->rc, "%s", r->err.c_str());
    if (r->collected) return set_error(HWC_ERR_STATE, "result of %llu already collected", (unsigned long long)ticket);
    r->collected = true;
    *out = r->result;
    r->result = nullptr;
    return HWC_OK;
}

extern "C" int hwc_serve_latency(hwc_server_t *s, uint64_t ticket, double *queued_us, double *total_us)
{
    if (!s) return set_error(HWC_ERR_ARG, "null argument");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) return set_error(HWC_ERR_ARG, "unknown ticket");
    Request *r = it->second;
    if (r->state != 2) return set_error(HWC_ERR_STATE, "request not finished");
    using us = std::chrono::duration<double, std::micro>;
    if (queued_us) *queued_us = r->rc ? 0.0 : us(r->t_admit - r->t_submit).count();
    if (total_us) *total_us = us(r->t_done - r->t_submit).count();
    return HWC_OK;
}

extern "C" int hwc_serve_close(hwc_server_t *s)
{
    if (!s) return HWC_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->th.joinable()) s->th.join();
    for (auto &kv : s->all) {
        free_request_device(kv.second);
        hwc_hist_free(kv.second->result);
        delete kv.second;
    }
    cudaFree(s->d_jobs);
    cudaFree(s->d_item_start);
    cudaFree(s->d_counters);
    cudaFree(s->d_wkeys);
    if (s->h_jobs) cudaFreeHost(s->h_jobs);
    if (s->h_item_start) cudaFreeHost(s->h_item_start);
    if (s->stream) cudaStreamDestroy(s->stream);
    delete s;
    return HWC_OK;
}
