// serve.cu -- request loop with continuous batching.
//
// A server thread owns two CUDA streams and runs the device in steps.  Each
// step is one launch of the persistent count kernel per kernel group over a
// slice of every active request (an equal share of point evaluations each,
// about kStepMs of device time in all at the rate measured on earlier steps),
// so requests of very different sizes progress together, and a request that
// arrives while others run joins at the next step once a slot and enough
// device memory are free.  The host never waits for the step it has just
// enqueued: step i+1 is built and enqueued while step i runs, and only then
// does the thread wait for step i and hand out the results of the requests
// it finished.  Per-request memory comes from the stream-ordered allocator
// and is cleared, compacted and released on the second stream, so admission
// and completion do not synchronise the device either.  Field tables stay
// resident in the process-wide table cache.  Each request owns its histogram
// hash; slices of one request add into it across steps.  Results do not
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
    KJob *d_one = nullptr;   // device copy of kj (clear, compact)
    uint64_t next_tile = 0;
    std::vector<void *> allocs;
    uint64_t bytes = 0;
    int state = 0;   // 0 queued, 1 active, 2 done
    int rc = HWC_OK;
    std::string err;
    hwc_hist *result = nullptr;
    // the compacted (key, count) list copied back; the sorted histogram is
    // built from it in the thread that collects the result
    std::vector<unsigned long long> rkeys, rcnt;
    uint64_t rtotal = 0;
    bool collected = false;
    Clock::time_point t_submit, t_admit, t_done;
};

// a step on the device whose results are not yet handed out
struct Inflight {
    bool valid = false;
    std::vector<Request *> reqs;
    std::vector<uint64_t> took;
    std::vector<Request *> finishing;   // requests whose last tiles the step runs
    double evals = 0;
    int rc = HWC_OK;
};

}  // namespace

struct hwc_server {
    hwc_server_config_t cfg{};
    int device = 0;
    cudaStream_t stream = nullptr;   // steps
    cudaStream_t aux = nullptr;      // per-request allocation, clearing, compaction, release
    std::thread th;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request *> pending;
    std::vector<Request *> active;
    uint32_t retiring = 0;           // requests whose last step is still in flight
    std::map<uint64_t, Request *> all;
    uint64_t next_ticket = 1;
    bool stop = false;
    uint64_t used_bytes = 0;
    std::set<std::pair<uint32_t, uint32_t>> tables_seen;
    KJob *d_jobs = nullptr;
    uint64_t *d_item_start = nullptr;     // [2 * max_active]
    unsigned long long *d_counters = nullptr;   // [max_active]
    KJob *h_jobs[2] = {};            // pinned staging, one per step in flight
    uint64_t *h_item_start[2] = {};
    cudaEvent_t ev_t0[2] = {}, ev_t1[2] = {};
    cudaEvent_t ev_admit = nullptr;
    cudaMemPool_t pool = nullptr;    // per-request memory (kept mapped between requests)
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

// point evaluations of one tile of a job: members per tile (q^2 for the
// two-level fan-out, q for the c_0 fan-out, 32 per member tile) times the
// points the kernels evaluate per member (one per Frobenius orbit)
double tile_evals(const KJob &kj)
{
    const double members = kj.method == 2 ? (double)kj.q * kj.q : (kj.method == 1 ? (double)kj.q : (double)kTileMembers);
    double pts = 0;
    for (uint32_t k = 0; k < kj.g; ++k) pts += kj.npts[k] + 1;
    return members * pts;
}

void free_request_device(hwc_server *s, Request *r)
{
    for (void *p : r->allocs) cudaFreeAsync(p, s->aux);
    r->allocs.clear();
}

// one stream-ordered allocation per request, carved into its arrays
int ralloc_all(hwc_server *s, Request *r, const uint64_t *bytes, void **ptrs, int n)
{
    uint64_t total = 0, off[16];
    for (int i = 0; i < n; ++i) {
        off[i] = total;
        total += (bytes[i] + 255) / 256 * 256;
    }
    void *v = nullptr;
    if (cudaMallocFromPoolAsync(&v, total, s->pool, s->aux) != cudaSuccess) {
        cudaGetLastError();
        return set_error(HWC_ERR_NOMEM, "cudaMallocFromPoolAsync of %llu bytes failed", (unsigned long long)total);
    }
    r->allocs.push_back(v);
    for (int i = 0; i < n; ++i) ptrs[i] = (char *)v + off[i];
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

// admission (server thread): the request's hash, allocated and cleared on the
// second stream; the step stream waits for it before its next launch
int admit(hwc_server *s, Request *r)
{
    KJob &kj = r->kj;
    const uint64_t cap = kj.hmask + 1ull;
    const uint64_t bytes[8] = {8 * cap, 8 * cap, 8 * 4, 8 * cap, 8 * cap, 8, sizeof(KJob),
                               needs_weights(kj) ? 4 * kj.w_n : 0};
    void *ptrs[8];
    int rc = ralloc_all(s, r, bytes, ptrs, 8);
    if (rc) return rc;
    if (needs_weights(kj)) kj.mweight = (uint32_t *)ptrs[7];
    kj.hkeys = (unsigned long long *)ptrs[0];
    kj.hcounts = (unsigned long long *)ptrs[1];
    kj.stats = (unsigned long long *)ptrs[2];
    kj.out_keys = (unsigned long long *)ptrs[3];
    kj.out_counts = (unsigned long long *)ptrs[4];
    kj.n_out = (unsigned long long *)ptrs[5];
    r->d_one = (KJob *)ptrs[6];
    HWC_CUDA_TRY(cudaMemcpyAsync(r->d_one, &kj, sizeof kj, cudaMemcpyHostToDevice, s->aux));
    rc = launch_clear(r->d_one, 1, nullptr, 0, s->aux);
    if (rc) return rc;
    if ((rc = launch_sample_weights(kj, s->aux))) return rc;   // the samples' multiplicities
    HWC_CUDA_TRY(cudaEventRecord(s->ev_admit, s->aux));
    HWC_CUDA_TRY(cudaStreamWaitEvent(s->stream, s->ev_admit, 0));
    return HWC_OK;
}

// finished request (its last step is complete): compact its hash on the second
// stream and copy the (key, count) list back
int finish(hwc_server *s, Request *r)
{
    int rc = launch_compact(r->d_one, 1, s->aux);
    if (rc) return rc;
    unsigned long long st[3] = {}, n_out = 0;
    HWC_CUDA_TRY(cudaMemcpyAsync(st, r->kj.stats, sizeof st, cudaMemcpyDeviceToHost, s->aux));
    HWC_CUDA_TRY(cudaMemcpyAsync(&n_out, r->kj.n_out, sizeof n_out, cudaMemcpyDeviceToHost, s->aux));
    HWC_CUDA_TRY(cudaStreamSynchronize(s->aux));
    if (st[2]) return set_error(HWC_ERR_TOO_LARGE, "histogram hash overflowed");
    r->rkeys.resize(n_out);
    r->rcnt.resize(n_out);
    if (n_out) {
        HWC_CUDA_TRY(cudaMemcpyAsync(r->rkeys.data(), r->kj.out_keys, n_out * 8, cudaMemcpyDeviceToHost, s->aux));
        HWC_CUDA_TRY(cudaMemcpyAsync(r->rcnt.data(), r->kj.out_counts, n_out * 8, cudaMemcpyDeviceToHost, s->aux));
        HWC_CUDA_TRY(cudaStreamSynchronize(s->aux));
    }
    r->rtotal = st[0];
    return HWC_OK;
}

void complete(hwc_server *s, Request *r, int rc)
{
    // called with s->mu held
    r->rc = rc;
    if (rc) r->err = hwc_last_error();
    r->state = 2;
    r->t_done = Clock::now();
    free_request_device(s, r);
    s->used_bytes -= std::min(s->used_bytes, r->bytes);
    s->cv_done.notify_all();
}

// Build one step over `step` (a slice of every request) into staging buffer
// `buf` and enqueue it on the step stream; requests of one kernel group share
// a persistent launch.  Advances each request's next tile.
int enqueue_step(hwc_server *s, std::vector<Request *> &step, int buf, Inflight &inf)
{
    auto skey = [](const Request *x) { return std::make_tuple(x->kj.d, x->kj.method, x->kj.words); };
    std::stable_sort(step.begin(), step.end(), [&](const Request *x, const Request *y) { return skey(x) < skey(y); });
    const uint32_t n = (uint32_t)step.size();
    inf.reqs = step;
    inf.took.assign(n, 0);
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
    KJob *hj = s->h_jobs[buf];
    uint64_t *hs = s->h_item_start[buf];
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
            if (rc == HWC_OK && (uint64_t)G.sh.grid * (G.sh.block / 32) * 961ull > s->wkeys_slots)
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
            if (!s->cfg.step_items) want = std::max<uint64_t>(want, (uint64_t)(req_evals / tile_evals(q->kj)) + 1);
            const uint64_t t = std::min(left, want);
            inf.took[r] = t;
            inf.evals += (double)t * tile_evals(q->kj);
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
            hj[r] = sl;
            hs[item_off + (r - i)] = items;
            items += (t + G.sh.item_tiles - 1) / G.sh.item_tiles;
        }
        hs[item_off + (e - i)] = items;
        G.items = items;
        item_off += (e - i) + 1;
        groups.push_back(G);
        ++ngroups;
        i = e;
    }
    if (rc) return rc;
    // descriptors from pinned memory, then the launches, all on the step stream
    HWC_CUDA_TRY(cudaMemcpyAsync(s->d_jobs, hj, n * sizeof(KJob), cudaMemcpyHostToDevice, s->stream));
    HWC_CUDA_TRY(cudaMemcpyAsync(s->d_item_start, hs, item_off * sizeof(uint64_t), cudaMemcpyHostToDevice, s->stream));
    HWC_CUDA_TRY(cudaMemsetAsync(s->d_counters, 0, ngroups * sizeof(unsigned long long), s->stream));
    HWC_CUDA_TRY(cudaEventRecord(s->ev_t0[buf], s->stream));
    for (size_t g = 0; g < groups.size(); ++g) {
        const StepGroup &G = groups[g];
        rc = launch_persistent(G.D, G.method, G.words, s->d_jobs + G.first, s->d_item_start + G.off, G.n, G.items,
                               s->d_counters + g, G.smem, G.sh, s->stream);
        if (rc) return rc;
    }
    HWC_CUDA_TRY(cudaEventRecord(s->ev_t1[buf], s->stream));
    for (uint32_t i = 0; i < n; ++i) {
        Request *r = step[i];
        r->next_tile += inf.took[i];
        if (r->next_tile >= r->kj.n_tiles) inf.finishing.push_back(r);
    }
    return HWC_OK;
}

// wait for a step in flight and hand out the requests it finished
void retire_step(hwc_server *s, Inflight &inf, int buf)
{
    int rc = inf.rc;
    if (rc == HWC_OK) {
        cudaError_t ce = cudaEventSynchronize(s->ev_t1[buf]);
        if (ce != cudaSuccess) rc = set_error(HWC_ERR_CUDA, "step: %s", cudaGetErrorString(ce));
    }
    if (rc == HWC_OK) {   // the step's device rate updates the running mean
        float ms = 0;
        if (cudaEventElapsedTime(&ms, s->ev_t0[buf], s->ev_t1[buf]) == cudaSuccess && ms > 0 && inf.evals > 0)
            s->evals_per_ms = s->evals_per_ms > 0 ? 0.5 * s->evals_per_ms + 0.5 * (inf.evals / ms) : inf.evals / ms;
    }
    if (rc) {   // nothing may still run on a request's memory when it is released
        cudaStreamSynchronize(s->stream);
        cudaGetLastError();
    }
    std::vector<int> frc(inf.finishing.size(), rc);
    if (rc == HWC_OK)
        for (size_t i = 0; i < inf.finishing.size(); ++i) frc[i] = finish(s, inf.finishing[i]);
    std::lock_guard<std::mutex> lk(s->mu);
    if (rc) {   // a failed step fails every request it touched
        for (Request *r : inf.reqs) {
            if (r->state == 2) continue;
            s->active.erase(std::remove(s->active.begin(), s->active.end(), r), s->active.end());
            complete(s, r, rc);
        }
    }
    for (size_t i = 0; i < inf.finishing.size(); ++i)
        if (inf.finishing[i]->state != 2) complete(s, inf.finishing[i], frc[i]);
    s->retiring -= std::min<uint32_t>(s->retiring, (uint32_t)inf.finishing.size());
    inf = Inflight();
}

void server_loop(hwc_server *s)
{
    cudaSetDevice(s->device);
    const uint32_t max_active = std::max<uint32_t>(1, s->cfg.max_active);
    Inflight prev;
    int buf = 0;
    for (;;) {
        std::vector<Request *> step;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            for (;;) {
                // admit while a slot and memory are free
                while (!s->pending.empty() && s->active.size() + s->retiring < max_active) {
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
                if (!s->active.empty() || prev.valid) break;
                if (s->stop && s->pending.empty()) return;
                s->cv_work.wait(lk);
            }
            step = s->active;
        }
        // enqueue the next step while the previous one runs
        Inflight cur;
        if (!step.empty()) {
            cur.valid = true;
            cur.rc = enqueue_step(s, step, buf, cur);
            std::lock_guard<std::mutex> lk(s->mu);
            if (cur.rc) {
                cur.finishing.clear();
            } else {
                for (Request *r : cur.finishing)
                    s->active.erase(std::remove(s->active.begin(), s->active.end(), r), s->active.end());
                s->retiring += (uint32_t)cur.finishing.size();
            }
            ++s->steps;
        }
        if (prev.valid) retire_step(s, prev, buf ^ 1);
        if (cur.valid && cur.rc) {   // nothing of it runs: fail its requests now
            retire_step(s, cur, buf);
            continue;
        }
        prev = cur;
        buf ^= 1;
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
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = s->device;
    const uint64_t keep = ~0ull;   // keep freed request memory mapped for the next requests
    bool ok = cudaMemPoolCreate(&s->pool, &props) == cudaSuccess &&
              cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, (void *)&keep) == cudaSuccess &&
              cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&s->aux, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&s->ev_admit, cudaEventDisableTiming) == cudaSuccess &&
              cudaMalloc(&s->d_jobs, m * sizeof(KJob)) == cudaSuccess &&
              cudaMalloc(&s->d_item_start, 2 * (m + 1) * sizeof(uint64_t)) == cudaSuccess &&
              cudaMalloc(&s->d_counters, m * sizeof(unsigned long long)) == cudaSuccess;
    for (int b = 0; b < 2 && ok; ++b)
        ok = cudaMallocHost(&s->h_jobs[b], m * sizeof(KJob)) == cudaSuccess &&
             cudaMallocHost(&s->h_item_start[b], 2 * (m + 1) * sizeof(uint64_t)) == cudaSuccess &&
             cudaEventCreate(&s->ev_t0[b]) == cudaSuccess && cudaEventCreate(&s->ev_t1[b]) == cudaSuccess;
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
    int rc = fill_kjob(*job, r->kj, &fam_n, kFlagNoClass, &tc);   // validates, builds tables
    if (rc) {
        delete r;
        return rc;
    }
    r->kj.hmask = hash_capacity(r->kj.g, r->kj.q, job->count, 1) - 1;
    r->bytes = 32ull * (r->kj.hmask + 1ull) + 4096 + (needs_weights(r->kj) ? 4 * r->kj.w_n : 0);
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
    // the sorted histogram, built here in the caller's thread (not the server's)
    std::vector<unsigned long long> keys, cnt;
    keys.swap(r->rkeys);
    cnt.swap(r->rcnt);
    const KJob kj = r->kj;
    const uint64_t total = r->rtotal;
    lk.unlock();
    *out = hist_from_keys(kj, keys.data(), cnt.data(), keys.size(), total);
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
        if (s->aux) free_request_device(s, kv.second);
        hwc_hist_free(kv.second->result);
        delete kv.second;
    }
    if (s->aux) cudaStreamSynchronize(s->aux);
    if (s->stream) cudaStreamSynchronize(s->stream);
    cudaFree(s->d_jobs);
    cudaFree(s->d_item_start);
    cudaFree(s->d_counters);
    cudaFree(s->d_wkeys);
    for (int b = 0; b < 2; ++b) {
        if (s->h_jobs[b]) cudaFreeHost(s->h_jobs[b]);
        if (s->h_item_start[b]) cudaFreeHost(s->h_item_start[b]);
        if (s->ev_t0[b]) cudaEventDestroy(s->ev_t0[b]);
        if (s->ev_t1[b]) cudaEventDestroy(s->ev_t1[b]);
    }
    if (s->ev_admit) cudaEventDestroy(s->ev_admit);
    if (s->stream) cudaStreamDestroy(s->stream);
    if (s->aux) cudaStreamDestroy(s->aux);
    if (s->pool) cudaMemPoolDestroy(s->pool);
    delete s;
    return HWC_OK;
}
