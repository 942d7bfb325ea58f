// count_kernels.cu -- launch wrappers of the count kernels, the histogram
// clear/compaction kernels, and the allocation-free entry point.  The
// per-member Horner kernels are in horner.cuh (instantiated in horner_*.cu),
// the c_0 fan-out kernels in fanout.cuh (fanout_*.cu).
#include "count_common.cuh"

#include <algorithm>
#include <cstring>

namespace hwc {
namespace {

__global__ void k_clear(const KJob *__restrict__ jobs, uint32_t n_jobs, unsigned long long *counters,
                        uint32_t n_counters)
{
    const uint32_t jb = blockIdx.y;
    if (jb == 0 && blockIdx.x == 0 && counters)
        for (uint32_t i = threadIdx.x; i < n_counters; i += blockDim.x) counters[i] = 0;
    if (jb >= n_jobs) return;
    const KJob &J = jobs[jb];
    if (blockIdx.x == 0 && threadIdx.x < 4) {
        if (threadIdx.x < 3) J.stats[threadIdx.x] = 0;
        else if (J.n_out) *J.n_out = 0;
    }
    if (!J.hkeys) return;
    const uint64_t cap = (uint64_t)J.hmask + 1;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cap;
         i += (uint64_t)gridDim.x * blockDim.x) {
        J.hkeys[i] = kEmptyKey;
        J.hcounts[i] = 0;
    }
}

__global__ void k_compact(const KJob *__restrict__ jobs, uint32_t n_jobs)
{
    const uint32_t jb = blockIdx.y;
    if (jb >= n_jobs) return;
    const KJob &J = jobs[jb];
    if (!J.hkeys) return;
    const uint64_t cap = (uint64_t)J.hmask + 1;
    const int lane = threadIdx.x & 31;
    for (uint64_t base = (uint64_t)blockIdx.x * blockDim.x; base < cap;
         base += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t i = base + threadIdx.x;
        const bool full = i < cap && J.hkeys[i] != kEmptyKey;
        const unsigned bal = __ballot_sync(kFull, full);
        unsigned long long pos = 0;
        if (lane == 0 && bal) pos = atomicAdd(J.n_out, (unsigned long long)__popc(bal));
        pos = __shfl_sync(kFull, pos, 0);
        if (full) {
            const uint64_t o = pos + __popc(bal & ((1u << lane) - 1u));
            J.out_keys[o] = J.hkeys[i];
            J.out_counts[o] = J.hcounts[i];
        }
    }
}

// multiplicities of the sampled members (the choice of f in Algorithm 1 for
// a sampled family, hwc.h): sample j draws member floor(z_j * fam / 2^64)
// (members w_first <= idx < w_first + w_n kept, at w[idx - w_first])
__global__ void k_sample_weights(uint64_t seed, uint64_t s_first, uint64_t s_count, uint64_t fam,
                                 uint64_t w_first, uint64_t w_n, uint32_t *__restrict__ w)
{
    for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < s_count;
         j += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t idx = __umul64hi(splitmix64_at(seed, s_first + j), fam);
        if (idx - w_first < w_n) atomicAdd(w + (idx - w_first), 1u);   // unsigned: idx >= w_first too
    }
}

// Counting sort of a class-sharing job's samples by class c = idx / q^2 (the
// digits c_2..c_{d-2} of member idx): per-class counts, then one CTA turns
// them into class starts (cnt[c] becomes the cursor) and writes the tile list
// (up to 32 samples of one class per tile), then every sample is placed by an
// atomic on its class cursor, which ends at the end of the class.
__global__ void k_cls_count(uint64_t seed, uint64_t first, uint64_t count, uint64_t fam, uint64_t q2,
                            uint32_t *__restrict__ cnt)
{
    for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < count;
         j += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t idx = __umul64hi(splitmix64_at(seed, first + j), fam);
        atomicAdd(cnt + idx / q2, 1u);
    }
}

constexpr int kScanThreads = 1024;

__global__ void __launch_bounds__(kScanThreads) k_cls_scan(uint32_t *__restrict__ cnt, uint32_t n_cls,
                                                           uint2 *__restrict__ tiles, uint64_t n_tiles)
{
    __shared__ uint32_t s_n[kScanThreads / 32], s_t[kScanThreads / 32];
    __shared__ uint32_t s_total;
    const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
    const uint32_t per = (n_cls + kScanThreads - 1) / kScanThreads;
    const uint32_t a = min(n_cls, tid * per), b = min(n_cls, a + per);
    uint32_t sn = 0, st = 0;   // samples and tiles of this thread's classes
    for (uint32_t c = a; c < b; ++c) {
        sn += cnt[c];
        st += (cnt[c] + 31u) / 32u;
    }
    // block-wide exclusive scan of (sn, st)
    uint32_t in = sn, it = st;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t vn = __shfl_up_sync(0xFFFFFFFFu, in, o), vt = __shfl_up_sync(0xFFFFFFFFu, it, o);
        if ((int)lane >= o) {
            in += vn;
            it += vt;
        }
    }
    if (lane == 31) {
        s_n[warp] = in;
        s_t[warp] = it;
    }
    __syncthreads();
    if (warp == 0) {
        uint32_t wn = s_n[lane], wt = s_t[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t vn = __shfl_up_sync(0xFFFFFFFFu, wn, o), vt = __shfl_up_sync(0xFFFFFFFFu, wt, o);
            if ((int)lane >= o) {
                wn += vn;
                wt += vt;
            }
        }
        s_n[lane] = wn;   // inclusive over warps
        s_t[lane] = wt;
        if (lane == 31) s_total = wt;
    }
    __syncthreads();
    uint32_t off = in - sn + (warp ? s_n[warp - 1] : 0u);
    uint32_t toff = it - st + (warp ? s_t[warp - 1] : 0u);
    for (uint32_t c = a; c < b; ++c) {
        const uint32_t n = cnt[c];
        cnt[c] = off;   // the class cursor starts at the class start
        for (uint32_t r = 0; r < n; r += 32) tiles[toff++] = make_uint2(c, off + r);
        off += n;
    }
    for (uint64_t t = s_total + tid; t < n_tiles; t += kScanThreads) tiles[t] = make_uint2(0xFFFFFFFFu, 0u);
}

__global__ void k_cls_scatter(uint64_t seed, uint64_t first, uint64_t count, uint64_t fam, uint64_t q2,
                              uint32_t *__restrict__ cursor, uint32_t *__restrict__ sorted)
{
    for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < count;
         j += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t idx = __umul64hi(splitmix64_at(seed, first + j), fam);
        const uint64_t c = idx / q2;
        const uint32_t pos = atomicAdd(cursor + c, 1u);
        sorted[pos] = (uint32_t)(idx - c * q2);   // c_0 + c_1 q
    }
}

}  // namespace

int launch_class_sort(const KJob &kj, cudaStream_t s)
{
    if (!kj.cls_n || !kj.count) return HWC_OK;
    const uint64_t q2 = (uint64_t)kj.q * kj.q;
    const uint64_t want = (kj.count + 255) / 256;
    const unsigned grid = (unsigned)std::min<uint64_t>(want, (uint64_t)device_sm_count() * 8);
    HWC_CUDA_TRY(cudaMemsetAsync(kj.cls_cnt, 0, (size_t)kj.cls_n * sizeof(uint32_t), s));
    k_cls_count<<<grid, 256, 0, s>>>(kj.seed, kj.first, kj.count, kj.fam_mz, q2, kj.cls_cnt);
    HWC_CUDA_TRY(cudaGetLastError());
    k_cls_scan<<<1, kScanThreads, 0, s>>>(kj.cls_cnt, kj.cls_n, kj.cls_tiles, kj.n_tiles);
    HWC_CUDA_TRY(cudaGetLastError());
    k_cls_scatter<<<grid, 256, 0, s>>>(kj.seed, kj.first, kj.count, kj.fam_mz, q2, kj.cls_cnt, kj.cls_sorted);
    HWC_CUDA_TRY(cudaGetLastError());
    return HWC_OK;
}

int launch_sample_weights(const KJob &kj, cudaStream_t s)
{
    if (!kj.mweight) return HWC_OK;
    HWC_CUDA_TRY(cudaMemsetAsync(kj.mweight, 0, kj.w_n * sizeof(uint32_t), s));
    if (kj.s_count) {
        const uint64_t want = (kj.s_count + 255) / 256;
        const unsigned grid = (unsigned)std::min<uint64_t>(want, (uint64_t)device_sm_count() * 8);
        k_sample_weights<<<grid, 256, 0, s>>>(kj.seed, kj.s_first, kj.s_count, kj.fam_mz, kj.w_first, kj.w_n,
                                              kj.mweight);
        HWC_CUDA_TRY(cudaGetLastError());
    }
    return HWC_OK;
}

// ---------------------------------------------------------------------
// host launch wrappers

using KernelFn = const void *;

KernelFn horner_kernel(int D, int which)
{
    return D <= 6 ? horner_kernel_a(D, which) : D <= 8 ? horner_kernel_b(D, which) : horner_kernel_c(D, which);
}

KernelFn fan_kernel(int D, int W, bool persistent)
{
    if (W != 1 && W != 2) return nullptr;
    switch (D) {
    case 3: case 4: return fan_kernel_a(D, W, persistent);
    case 5: return fan_kernel_b(D, W, persistent);
    case 6: return fan_kernel_c(D, W, persistent);
    case 7: return fan_kernel_d(D, W, persistent);
    case 8: return fan_kernel_f(D, W, persistent);
    case 9: case 10: return fan_kernel_e(D, W, persistent);
    default: return nullptr;
    }
}

KernelFn fan2_kernel(int D, bool weighted)
{
    if (weighted) return D <= 6 ? fan2_kernel_wa(D) : fan2_kernel_wb(D);
    return D <= 6 ? fan2_kernel_a(D) : fan2_kernel_b(D);
}

static KernelFn persistent_fn(int D, int block = 256)
{
    return horner_kernel(D, block > 256 ? 3 : 1);
}

static KernelFn cls_fn(int D, int block = 256)
{
    return D >= 3 && D <= 6 ? cls_kernel_a(D, block > 256 ? 3 : 1) : nullptr;
}

int prepare_count_kernels(void)
{
    static std::mutex mu;
    static bool done[64] = {};
    int dev = 0;
    HWC_CUDA_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(mu);
    if (dev >= 0 && dev < 64 && done[dev]) return HWC_OK;
    const int optin = (int)device_smem_optin();
    for (int D = 3; D <= kMaxD; ++D) {
        for (KernelFn fn : {persistent_fn(D), persistent_fn(D, 768), fan_kernel(D, 1, true), fan_kernel(D, 2, true),
                            fan2_kernel(D, false), fan2_kernel(D, true), cls_fn(D), cls_fn(D, 768)}) {
            if (!fn) continue;   // no kernel for this degree and row width
            cudaFuncAttributes fa{};
            HWC_CUDA_TRY(cudaFuncGetAttributes(&fa, fn));   // static smem counts against the limit
            HWC_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              optin - (int)fa.sharedSizeBytes));
        }
    }
    if (dev >= 0 && dev < 64) done[dev] = true;
    return HWC_OK;
}

int device_sm_count(void)
{
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

uint32_t device_smem_optin(void)
{
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return n > 0 ? (uint32_t)n : 48u * 1024u;
}

// the per-member kernel has two instantiations: up to 256 threads per CTA, and
// up to 768 (chosen by the block size)
static KernelFn kernel_for(int D, uint32_t method, uint32_t words, bool persistent, int block)
{
    if (method == 2) return fan2_kernel(D, words == 2);   // words 2: the weighted (sampled) variant
    if (method == 1) return fan_kernel(D, (int)words, persistent);
    (void)persistent;   // every run is a persistent launch (a plain run has one job per launch)
    if (words == 1) return cls_fn(D, block);   // method 0, words 1: the class-sharing variant
    return persistent_fn(D, block);
}

int max_ctas_per_sm(int D, uint32_t method, uint32_t words, int block, uint32_t smem_bytes,
                    bool persistent, int *out)
{
    int n = 0;
    KernelFn fn = kernel_for(D, method, words, true, block);
    if (!fn) return set_error(HWC_ERR_ARG, "degree %d has no kernel", D);
    cudaFuncAttributes fa{};
    HWC_CUDA_TRY(cudaFuncGetAttributes(&fa, fn));
    if (block > fa.maxThreadsPerBlock) {   // above the kernel's launch bound
        *out = 0;
        return HWC_OK;
    }
    HWC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, block, smem_bytes));
    *out = n;
    return HWC_OK;
}

int launch_clear(const KJob *d_jobs, uint32_t n_jobs, unsigned long long *d_counters,
                 uint32_t n_counters, cudaStream_t s)
{
    dim3 grid(device_sm_count(), std::max<uint32_t>(n_jobs, 1));
    k_clear<<<grid, 256, 0, s>>>(d_jobs, n_jobs, d_counters, n_counters);
    HWC_CUDA_TRY(cudaGetLastError());
    return HWC_OK;
}

int launch_persistent(int D, uint32_t method, uint32_t words, const KJob *d_jobs,
                      const uint64_t *d_item_start, uint32_t n_jobs, uint64_t n_items,
                      unsigned long long *d_counter, uint32_t max_smem, const LaunchShape &sh,
                      cudaStream_t s)
{
    KernelFn fn = kernel_for(D, method, words, true, sh.block);
    if (!fn) return set_error(HWC_ERR_ARG, "degree %d has no kernel", D);
    uint32_t item_tiles = (uint32_t)sh.item_tiles;
    void *args[] = {(void *)&d_jobs, (void *)&d_item_start, (void *)&n_jobs, (void *)&n_items,
                    (void *)&d_counter, (void *)&item_tiles};
    HWC_CUDA_TRY(cudaLaunchKernel(fn, dim3(sh.grid), dim3(sh.block), args, max_smem, s));
    return HWC_OK;
}

int launch_compact(const KJob *d_jobs, uint32_t n_jobs, cudaStream_t s)
{
    dim3 grid(device_sm_count(), std::max<uint32_t>(n_jobs, 1));
    k_compact<<<grid, 256, 0, s>>>(d_jobs, n_jobs);
    HWC_CUDA_TRY(cudaGetLastError());
    return HWC_OK;
}

}  // namespace hwc

// ---------------------------------------------------------------------
// Histogram without device allocation (hwc_count_noalloc).
//
// Some callers cannot call cudaMalloc when they count: processes that reserve
// all device memory up front and hand out fixed pools, threads that must not
// block on the device-wide synchronisation cudaMalloc implies, or host
// applications whose plug-in rules forbid device allocation.  This entry point keeps all of its working memory in one
// file-scope device array of fixed size: the histogram hash (keys and
// counts), the member statistics and the entry counter.  The job descriptor
// travels as a kernel parameter, the field tables are the caller's handles
// built earlier, and the results go to device buffers the caller owns.

namespace hwc {
namespace {

constexpr uint32_t kNoAllocSlots = 1u << 15;   // hash slots: distinct tuples < 16384
// layout: stats[4] | entries | pad[3] | keys[kNoAllocSlots] | counts[kNoAllocSlots]
constexpr size_t kNoAllocHeader = 8 * sizeof(unsigned long long);
constexpr size_t kNoAllocBytes = kNoAllocHeader + 2 * sizeof(unsigned long long) * kNoAllocSlots;

// one per device that loads the library; every call shares it
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

__global__ void k_na_clear(unsigned char *scratch, uint32_t slots)
{
    unsigned long long *hdr = reinterpret_cast<unsigned long long *>(scratch);
    unsigned long long *keys = hdr + 8;
    unsigned long long *cnts = keys + kNoAllocSlots;
    if (blockIdx.x == 0 && threadIdx.x < 8) hdr[threadIdx.x] = 0;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < slots; i += gridDim.x * blockDim.x) {
        keys[i] = kEmptyKey;
        cnts[i] = 0;
    }
}

// filled hash slots -> caller's (#C_1..#C_g, multiplicity) arrays, hash order
__global__ void k_na_emit(const KJob J, int32_t *counts, uint64_t *mult, uint64_t max_entries)
{
    unsigned long long *entries = J.stats + 4;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i <= J.hmask; i += gridDim.x * blockDim.x) {
        const unsigned long long key = J.hkeys[i];
        if (key == kEmptyKey) continue;
        const unsigned long long o = atomicAdd(entries, 1ull);
        if (o >= max_entries) continue;
        for (uint32_t k = 0; k < J.g; ++k) {
            const int a = (int)((key >> (16 * k)) & 0xFFFFu) - 32768;
            counts[o * J.g + k] = (int32_t)J.Q[k] + 1 - a;   // #C = Q + 1 - a (eq. 1.1)
        }
        mult[o] = J.hcounts[i];
    }
}

// n_out[0..2] = entries, square-free members, members examined
__global__ void k_na_finish(const KJob J, uint64_t *n_out)
{
    if (threadIdx.x == 0) {
        n_out[0] = J.stats[4];
        n_out[1] = J.stats[1];
        n_out[2] = J.stats[0];
    }
}

KernelFn na_count_kernel(int D)
{
    return horner_kernel(D, 2);
}

// Set-up, once per device with that device current: the device address of the
// scratch array (its name in host code is only a stand-in) and the kernels'
// shared-memory limit.
int noalloc_setup(unsigned char **scratch)
{
    static std::mutex mu;
    static unsigned char *addr[64] = {};
    int dev = 0;
    HWC_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return set_error(HWC_ERR_ARG, "device %d not supported", dev);
    std::lock_guard<std::mutex> lk(mu);
    if (!addr[dev]) {
        void *p = nullptr;
        HWC_CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        const int optin = (int)device_smem_optin();
        for (int D = 3; D <= kMaxD; ++D) {
            KernelFn fn = na_count_kernel(D);
            cudaFuncAttributes fa{};
            HWC_CUDA_TRY(cudaFuncGetAttributes(&fa, fn));
            HWC_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              optin - (int)fa.sharedSizeBytes));
        }
        addr[dev] = (unsigned char *)p;
    }
    *scratch = addr[dev];
    return HWC_OK;
}

}  // namespace
}  // namespace hwc

extern "C" int hwc_count_noalloc(uint32_t g, uint32_t q, const hwc_family_t *fam, uint64_t first,
                                 uint64_t count, const hwc_tables_t *const *tables, uint64_t max_entries,
                                 int32_t *counts, uint64_t *mult, uint64_t *n_out, void *stream)
{
    using namespace hwc;
    if (!fam || !tables || !n_out || (max_entries && (!counts || !mult)))
        return set_error(HWC_ERR_ARG, "null argument");
    if (g < 1 || g > (uint32_t)kMaxG) return set_error(HWC_ERR_ARG, "g=%u outside [1,%d]", g, kMaxG);
    const uint32_t d = fam->degree;
    if (d != 2 * g + 1 && d != 2 * g + 2) return set_error(HWC_ERR_ARG, "degree %u is not 2g+1 or 2g+2", d);
    if (fam->kind > HWC_FAM_MONIC_NOSUB_SAMPLED)
        return set_error(HWC_ERR_ARG, "family kind %u is not counted without allocation", fam->kind);
    uint64_t fam_n = 0;
    int rc = hwc_family_size(q, fam, &fam_n);
    if (rc) return rc;
    if (first > fam_n || count > fam_n - first)
        return set_error(HWC_ERR_RANGE, "members outside the family of %llu", (unsigned long long)fam_n);
    const uint32_t cap = hash_capacity(g, q, count, 1);
    if (cap > kNoAllocSlots)
        return set_error(HWC_ERR_TOO_LARGE, "histogram may need %u hash slots; the fixed scratch has %u", cap,
                         kNoAllocSlots);
    // job descriptor from the caller's tables (no table cache, no allocation)
    KJob kj;
    std::memset(&kj, 0, sizeof kj);
    uint32_t p = 0, e = 0;
    if (!prime_power(q, &p, &e)) return set_error(HWC_ERR_ARG, "q=%u is not an odd prime power", q);
    kj.g = g;
    kj.q = q;
    kj.d = d;
    kj.kind = fam->kind;
    kj.p = p;
    kj.seed = fam->seed;
    kj.first = first;
    kj.count = count;
    kj.fam_mz = 1;
    for (uint32_t i = 0; i + 1 < d; ++i) kj.fam_mz *= q;
    kj.qd = kj.fam_mz * q;
    kj.n_tiles = (count + kTileMembers - 1) / kTileMembers;
    int dev = 0;
    HWC_CUDA_TRY(cudaGetDevice(&dev));
    for (uint32_t k = 1; k <= g; ++k) {
        const hwc_tables_t *h = tables[k - 1];
        if (!h || !h->t || h->t->q != q || h->t->k != k)
            return set_error(HWC_ERR_ARG, "tables[%u] must be the tables of F_%u^%u", k - 1, q, k);
        // a handle built on another device holds that device's pointers
        if (h->t->device != dev)
            return set_error(HWC_ERR_ARG, "tables[%u] were built on device %d, the current device is %d", k - 1,
                             h->t->device, dev);
        const Tables *t = h->t;
        kj.Q[k - 1] = t->Q;
        kj.L[k - 1] = t->L;
        kj.barrett[k - 1] = (uint32_t)((1ull << 32) / t->L);
        kj.zech2[k - 1] = t->d_zech2;
        kj.zech3[k - 1] = t->d_zech3;
        kj.zech2w[k - 1] = t->d_zech2w;
        kj.coef_log[k - 1] = t->d_coef_log;
        kj.z17lo[k - 1] = t->d_z17lo;
        kj.z17hi[k - 1] = t->d_z17hi;
        set_points(kj, k, t, true);
    }
    layout_job_smem(kj, device_smem_optin() - 4096);
    unsigned char *scratch = nullptr;
    if ((rc = noalloc_setup(&scratch))) return rc;
    unsigned long long *hdr = reinterpret_cast<unsigned long long *>(scratch);
    kj.stats = hdr;                   // stats[0..3], entries at stats[4]
    kj.hkeys = hdr + 8;
    kj.hcounts = hdr + 8 + kNoAllocSlots;
    kj.hmask = cap - 1;
    cudaStream_t s = (cudaStream_t)stream;
    const int sms = device_sm_count();
    k_na_clear<<<sms, 256, 0, s>>>(scratch, cap);
    HWC_CUDA_TRY(cudaGetLastError());
    if (count) {
        int ctas = 0;
        KernelFn fn = na_count_kernel((int)d);
        HWC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ctas, fn, 256, kj.smem_bytes));
        if (ctas <= 0) return set_error(HWC_ERR_TOO_LARGE, "no CTA fits %u bytes of shared memory", kj.smem_bytes);
        const uint64_t need = (kj.n_tiles + 7) / 8;
        const int grid = (int)std::max<uint64_t>(1, std::min<uint64_t>(need, (uint64_t)sms * ctas));
        void *args[] = {(void *)&kj};
        HWC_CUDA_TRY(cudaLaunchKernel(fn, dim3(grid), dim3(256), args, kj.smem_bytes, s));
    }
    k_na_emit<<<sms, 256, 0, s>>>(kj, counts, mult, max_entries);
    HWC_CUDA_TRY(cudaGetLastError());
    k_na_finish<<<1, 32, 0, s>>>(kj, n_out);
    HWC_CUDA_TRY(cudaGetLastError());
    unsigned long long st[5] = {};
    HWC_CUDA_TRY(cudaMemcpyAsync(st, kj.stats, sizeof st, cudaMemcpyDeviceToHost, s));
    HWC_CUDA_TRY(cudaStreamSynchronize(s));
    if (st[2]) return set_error(HWC_ERR_TOO_LARGE, "histogram hash overflowed");
    if (st[4] > max_entries)
        return set_error(HWC_ERR_TOO_LARGE, "%llu histogram entries, output holds %llu",
                         (unsigned long long)st[4], (unsigned long long)max_entries);
    return HWC_OK;
}
