// tune.cu -- the autotuner.  Per class of jobs (device, g, q, degree, family
// kind and the flags that restrict the kernel) it times the candidate kernel
// choices -- per-member Horner (f-major), c_0 or (c_1, c_0) fan-out (x-major
// over groups of q or q^2 members), warps per CTA, tripled or doubled Zech
// tables in shared memory -- on a probe slice of the first job of the class
// and keeps the fastest.  Choices are cached per process and, when the
// environment variable HWC_TUNE_CACHE names a file, appended to that file and
// read back by later processes.  HWC_TUNE_VERBOSE=1 prints every timing.
#include "hwc_internal.cuh"

#include <cstdio>
#include <cstdlib>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

namespace hwc {
namespace {

using Key = std::tuple<int, uint32_t, uint32_t, uint32_t, uint32_t, uint32_t, uint32_t>;

std::mutex g_mu;
std::map<Key, TuneChoice> g_cache;
bool g_file_read = false;

constexpr uint32_t kFlagMask = HWC_FLAG_HORNER | HWC_FLAG_FAN1 | HWC_FLAG_ALL_POINTS | HWC_FLAG_LAMBDA;

Key key_of(const hwc_job_t &jb, uint32_t flags)
{
    return Key(device_sm_count(), device_smem_optin(), jb.g, jb.q, jb.family.degree, jb.family.kind,
               flags & kFlagMask);
}

void read_file_locked()
{
    if (g_file_read) return;
    g_file_read = true;
    const char *path = std::getenv("HWC_TUNE_CACHE");
    if (!path || !*path) return;
    FILE *f = std::fopen(path, "r");
    if (!f) return;
    int sms, method, warps, nt;
    unsigned optin, g, q, d, kind, fl;
    while (std::fscanf(f, "%d %u %u %u %u %u %u %d %d %d", &sms, &optin, &g, &q, &d, &kind, &fl, &method, &warps,
                       &nt) == 10) {
        TuneChoice c;
        c.method = method;
        c.warps = warps;
        c.no_triple = nt != 0;
        g_cache[Key(sms, optin, g, q, d, kind, fl)] = c;
    }
    std::fclose(f);
}

void append_file(const Key &k, const TuneChoice &c)
{
    const char *path = std::getenv("HWC_TUNE_CACHE");
    if (!path || !*path) return;
    FILE *f = std::fopen(path, "a");
    if (!f) return;
    std::fprintf(f, "%d %u %u %u %u %u %u %d %d %d\n", std::get<0>(k), std::get<1>(k), std::get<2>(k),
                 std::get<3>(k), std::get<4>(k), std::get<5>(k), std::get<6>(k), c.method, c.warps,
                 c.no_triple ? 1 : 0);
    std::fclose(f);
}

TuneChoice make(int method, int warps, bool no_triple)
{
    TuneChoice c;
    c.method = method;
    c.warps = warps;
    c.no_triple = no_triple;
    return c;
}

std::vector<TuneChoice> candidates(const hwc_job_t &jb, uint32_t flags)
{
    std::vector<TuneChoice> v;
    const bool sampled = jb.family.kind == HWC_FAM_MONIC_NOSUB_SAMPLED || jb.family.kind == HWC_FAM_REDUCED ||
                         jb.family.kind == HWC_FAM_MONIC_NOSUB_SAMPLED_WINDOW;
    if (sampled || (flags & (HWC_FLAG_HORNER | HWC_FLAG_LAMBDA)) || jb.q > 63) return {make(0, 0, false)};
    if (jb.q <= 31 && !(flags & HWC_FLAG_FAN1)) {
        v.push_back(make(2, 0, false));   // the default: most resident warps
        for (int w : {16, 8}) v.push_back(make(2, w, false));
        for (int w : {0, 16}) v.push_back(make(2, w, true));
    }
    v.push_back(make(1, 0, false));
    return v;
}

// members of the probe slice: about eight work items per resident warp, so
// that the tail of the launch weighs little
uint64_t probe_members(const hwc_job_t &jb, uint32_t flags)
{
    const uint64_t warps = (uint64_t)device_sm_count() * 24;
    const uint64_t q = jb.q;
    const uint64_t unit = (q <= 31 && !(flags & HWC_FLAG_FAN1)) ? q * q : q;
    return 8 * warps * unit;
}

bool verbose()
{
    const char *v = std::getenv("HWC_TUNE_VERBOSE");
    return v && *v && *v != '0';
}

// kernel time (ms) of one candidate on the probe, or a negative value
double time_candidate(const hwc_job_t &probe, const TuneChoice &c, uint32_t *method, uint32_t flags)
{
    hwc_batch *b = nullptr;
    if (batch_create_with(&probe, 1, HWC_FLAG_PLAIN | HWC_FLAG_TIMING | (flags & HWC_FLAG_ALL_POINTS), &c, &b) !=
        HWC_OK)
        return -1;
    double best = -1;
    hwc_batch_job_method(b, 0, method);
    for (int rep = 0; rep < 3; ++rep) {   // the first is a warm-up
        float ms = 0;
        if (hwc_batch_launch(b, nullptr) != HWC_OK || hwc_batch_kernel_ms(b, &ms) != HWC_OK) {
            best = -1;
            break;
        }
        if (rep > 0 && (best < 0 || ms < best)) best = ms;
    }
    hwc_batch_free(b);
    return best;
}

}  // namespace

bool tune_lookup(const hwc_job_t &jb, uint32_t flags, TuneChoice *out)
{
    std::lock_guard<std::mutex> lk(g_mu);
    read_file_locked();
    auto it = g_cache.find(key_of(jb, flags));
    if (it == g_cache.end()) return false;
    *out = it->second;
    return true;
}

int tune_choice(const hwc_job_t &jb, uint32_t flags, TuneChoice *out)
{
    *out = TuneChoice();
    if (tune_lookup(jb, flags, out)) return HWC_OK;
    const std::vector<TuneChoice> cand = candidates(jb, flags);
    if (cand.size() < 2) return HWC_OK;   // one kernel applies: nothing to measure
    const uint64_t want = probe_members(jb, flags);
    if (jb.count < want) return HWC_OK;   // too small to measure; left to the default rule, not cached
    // the middle of the job: the first members of a family have their high
    // coefficients zero (short chains), which would not be representative
    hwc_job_t probe = jb;
    probe.count = want;
    probe.first = jb.first + (jb.count - want) / 2;
    double best = -1;
    TuneChoice pick;
    std::vector<uint32_t> seen;   // (method, warps, no_triple) already timed
    for (const TuneChoice &c : cand) {
        uint32_t method = 0;
        const double ms = time_candidate(probe, c, &method, flags);
        if (ms < 0) {   // this candidate could not run (e.g. out of memory): skip it
            cudaGetLastError();
            continue;
        }
        if (verbose())
            std::fprintf(stderr, "hwc tune g=%u q=%u d=%u kind=%u: method %u warps %d %s -> %.3f ms\n", jb.g, jb.q,
                         jb.family.degree, jb.family.kind, method, c.warps, c.no_triple ? "doubled" : "tripled",
                         ms);
        const uint32_t tag = method * 1024 + (uint32_t)c.warps * 2 + (c.no_triple ? 1 : 0);
        bool dup = false;
        for (uint32_t t : seen) dup = dup || t == tag;
        if (dup) continue;
        seen.push_back(tag);
        // the candidates come in order of preference (the default first): a
        // later one must be more than 3% faster, not a timing fluctuation
        if (best < 0 || ms < 0.97 * best) {
            best = ms;
            pick = c;
            pick.method = (int)method;   // the kernel the choice ended up with
        }
    }
    if (best < 0) return HWC_OK;   // nothing measured: default rule
    *out = pick;
    std::lock_guard<std::mutex> lk(g_mu);
    const Key k = key_of(jb, flags);
    if (g_cache.emplace(k, pick).second) append_file(k, pick);
    return HWC_OK;
}

}  // namespace hwc
