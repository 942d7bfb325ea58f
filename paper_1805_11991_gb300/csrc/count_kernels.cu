// count_kernels.cu -- the point-counting hot path on sm_103a.
//
// One warp handles a tile of 32 consecutive members of a family:
//   1. each lane decodes one member index into coefficient digits (Algorithm 1
//      line 3) and tests it for square-freeness by Euclid's algorithm on
//      gcd(f, f') in Zech arithmetic over F_q;
//   2. for every square-free member of the tile (uniform loop) and every
//      k = 1..g the 32 lanes sweep x = alpha^j over F_Q^x (lines 6-14), two
//      x per lane per step, evaluating f by Horner's rule in the log domain
//      with one Zech lookup per nonzero coefficient (eq. 2.1, 3.1-3.2), and
//      sum chi(f(x)) = (-1)^log (the parity of the log, L being even);
//   3. #C_k = Q + sum_x chi(f(x)) + 1 + chi(f(inf)) (Sec. 1.1), i.e.
//      r^0 + 2 r^sq + 1 + chi(f(inf)); the lanes' tuples are aggregated
//      within the warp (match.any) and added into an open-addressing hash
//      in global memory (line 21, weight 1).
//
// The Horner chain is kept in "Zech index" form.  With lambda_i = log c_i and
// the nonzero coefficients below the lead at i_1 > i_2 > ..., the partial
// value after c_{i_t} is alpha^(lambda_{i_t} + Z(u_t)) and
//     u_{t+1} = Z(u_t) + (lambda_{i_t} - lambda_{i_{t+1}} + (i_t - i_{t+1}) j)  (mod L),
// so each step is one table read and a few integer adds.  The table is read
// through a doubled layout T[u] = Z(u mod L), u in [0, 2L), so u needs no
// reduction; the entry with 1 + alpha^u = 0 holds the poison value 2L, and
// T[2L] = 2L, so a vanishing partial sum (probability ~ 1/Q per step, Sec. 4)
// makes the chain stick at 2L; such lanes are redone by a branchy Horner.
#include "count_common.cuh"

#include <algorithm>
#include <cstring>

namespace hwc {
namespace {

template <int D, int I1, bool TRIPLE, class Tab>
__device__ __forceinline__ void dense_chain(const Tab T, const uint32_t (&dli)[D], uint32_t L,
                                            uint32_t cap, uint32_t xA, uint32_t xB,
                                            uint32_t &uA, uint32_t &uB)
{
#pragma unroll
    for (int i = I1 - 1; i >= 0; --i) {
        const uint32_t zA = T[uA], zB = T[uB];
        uA = chain_step<TRIPLE>(zA, dli[i], xA, L, cap);
        uB = chain_step<TRIPLE>(zB, dli[i], xB, L, cap);
    }
}

template <int D, bool TRIPLE, class Tab>
__device__ __forceinline__ int field_chi_sum(const Tab T, uint32_t L, uint32_t bar,
                                             const uint32_t (&lam)[D + 1], uint32_t nz, int lane)
{
    const uint32_t cap = TRIPLE ? 3 * L : 2 * L;
    int S = 0;
    if (nz == 0) {   // f = c_D x^D
        for (uint32_t j = lane; j < L; j += 32) S += ((lam[D] + (uint32_t)D * j) & 1u) ? -1 : 1;
        return S;
    }
    const int i1 = 31 - __clz(nz);
    const int is = __ffs(nz) - 1;
    const uint32_t g1 = (uint32_t)(D - i1);
    // first step index: lam_D + g1*j - lam_{i1}, kept in [0, 2L)
    const uint32_t base1 = lam[D] + (L - lam[i1]);     // < 2L
    const uint32_t lam_last = lam[is];
    const uint32_t is_odd = (uint32_t)is & 1u;
    // per-position constants of the chain (static indices: registers)
    uint32_t dli[D], gpi[D];
    {
        uint32_t lp = lam[i1];
        int ip = i1;
#pragma unroll
        for (int i = D - 1; i >= 0; --i) {
            dli[i] = 0;
            gpi[i] = 0;
            if (i < i1 && ((nz >> i) & 1u)) {
                dli[i] = addmod(lp, L - lam[i], L);
                gpi[i] = (uint32_t)(ip - i);
                lp = lam[i];
                ip = i;
            }
        }
    }
    // dense patterns get a branch-free chain
    const int dense = (nz == (1u << (D - 1)) - 1u) ? 2 : (nz == (1u << D) - 1u) ? 1 : 0;
    for (uint32_t j0 = 0; j0 < L; j0 += 64) {
        const uint32_t jA = j0 + lane, jB = j0 + 32 + lane;
        const bool vA = jA < L, vB = jB < L;
        const uint32_t xA = vA ? jA : 0, xB = vB ? jB : 0;
        uint32_t mA, mB;
        if (g1 == 2) {   // lead at D, first nonzero at D-2: 2j mod L
            mA = min(2 * xA, 2 * xA - L);
            mB = min(2 * xB, 2 * xB - L);
        } else {
            mA = mulmod_small(g1, xA, L, bar);
            mB = mulmod_small(g1, xB, L, bar);
        }
        uint32_t uA = base1 + mA, uB = base1 + mB;       // < 3L
        if (!TRIPLE) {
            uA = min(uA, uA - L);                          // unsigned: back below 2L
            uB = min(uB, uB - L);
        }
        if (dense == 2) {
            dense_chain<D, D - 2, TRIPLE>(T, dli, L, cap, xA, xB, uA, uB);
        } else if (dense == 1) {
            dense_chain<D, D - 1, TRIPLE>(T, dli, L, cap, xA, xB, uA, uB);
        } else {
#pragma unroll
            for (int i = D - 2; i >= 0; --i) {
                if (gpi[i] == 0) continue;                 // zero coefficient or above i1
                uint32_t sA, sB;
                if (gpi[i] == 1) {
                    sA = xA;
                    sB = xB;
                } else {
                    sA = mulmod_small(gpi[i], xA, L, bar);
                    sB = mulmod_small(gpi[i], xB, L, bar);
                }
                const uint32_t zA = T[uA], zB = T[uB];
                uA = chain_step<TRIPLE>(zA, dli[i], sA, L, cap);
                uB = chain_step<TRIPLE>(zB, dli[i], sB, L, cap);
            }
        }
        const uint32_t zA = T[uA], zB = T[uB];
        // f(x) = alpha^(lam_last + z + is*j): chi is the parity of the exponent
        int cA = 1 - 2 * (int)((lam_last ^ zA ^ (xA & is_odd)) & 1u);
        int cB = 1 - 2 * (int)((lam_last ^ zB ^ (xB & is_odd)) & 1u);
        const bool pA = vA && zA >= cap, pB = vB && zB >= cap;
        if (__any_sync(kFull, pA || pB)) {
            if (pA) cA = slow_chi<D>(T, L, cap, lam, nz, xA);
            if (pB) cB = slow_chi<D>(T, L, cap, lam, nz, xB);
        }
        S += (vA ? cA : 0) + (vB ? cB : 0);
    }
    return S;
}

// ---------------------------------------------------------------------
// one tile of 32 members, processed by one warp

template <int D>
__device__ void process_tile(const KJob &J, uint64_t tile, const uint8_t *smem, int lane,
                             WarpStats &st)
{
    constexpr int G = (D - 1) / 2;
    const uint64_t m = tile * kTileMembers + lane;
    const bool valid = m < J.count;
    uint32_t c[D + 1];
#pragma unroll
    for (int i = 0; i <= D; ++i) c[i] = 0;
    c[D] = 1;
    if (valid) decode_member<D>(J, m, c);

    const uint16_t *s16 = reinterpret_cast<const uint16_t *>(smem);
    const uint32_t *s32 = reinterpret_cast<const uint32_t *>(smem);

    bool sqf = false;
    if (valid) {
        const uint32_t *coef1 = s32 + J.coef_off[0];
        if (J.tab_kind[0] != kTabDoubleGlobal) {
            FqLog<TabS> F{TabS{s16 + J.tab_off[0]}, J.L[0]};
            sqf = squarefree<D>(F, coef1, J.p, c);
        } else {
            FqLog<TabG> F{TabG{J.zech2w[0]}, J.L[0]};
            sqf = squarefree<D>(F, coef1, J.p, c);
        }
    }
    const unsigned vmask = __ballot_sync(kFull, valid);
    const unsigned smask = __ballot_sync(kFull, sqf);
    if (lane == 0) {
        st.examined += __popc(vmask);
        st.sqf += __popc(smask);
    }
    unsigned todo = J.unfiltered ? vmask : smask;

    int32_t myN[G];
#pragma unroll
    for (int k = 0; k < G; ++k) myN[k] = 0;

    while (todo) {
        const int src = __ffs(todo) - 1;
        todo &= todo - 1;
        uint32_t cc[D + 1];
#pragma unroll
        for (int i = 0; i <= D; ++i) cc[i] = __shfl_sync(kFull, c[i], src);
        uint32_t nz = 0;
#pragma unroll
        for (int i = 0; i < D; ++i) nz |= (cc[i] != 0 ? 1u : 0u) << i;
#pragma unroll
        for (int k = 0; k < G; ++k) {
            const uint32_t L = J.L[k];
            const uint32_t *coefk = s32 + J.coef_off[k];
            uint32_t lam[D + 1];
#pragma unroll
            for (int i = 0; i <= D; ++i) lam[i] = coefk[cc[i]];
            int S;
            const uint32_t kind = J.tab_kind[k];
            if (kind == kTabTripleSmem)
                S = field_chi_sum<D, true>(TabS{s16 + J.tab_off[k]}, L, J.barrett[k], lam, nz, lane);
            else if (kind == kTabDoubleSmem)
                S = field_chi_sum<D, false>(TabS{s16 + J.tab_off[k]}, L, J.barrett[k], lam, nz, lane);
            else
                S = field_chi_sum<D, false>(TabG{J.zech2w[k]}, L, J.barrett[k], lam, nz, lane);
            if (lane == 0 && cc[0] != 0) S += (lam[0] & 1u) ? -1 : 1;   // x = 0
            S = __reduce_add_sync(kFull, S);
            // points at infinity: 1 + chi(c_{2g+2})
            int inf = 1;
            if (D == 2 * G + 2) inf += (lam[D] & 1u) ? -1 : 1;
            if (lane == src) myN[k] = (int32_t)J.Q[k] + S + inf;
        }
    }

    if (J.member_counts) {
        if (valid) {
#pragma unroll
            for (int k = 0; k < G; ++k) J.member_counts[m * G + k] = (sqf || J.unfiltered) ? myN[k] : 0;
            J.member_sqf[m] = sqf ? 1 : 0;
        }
        return;
    }
    unsigned long long key = 0;
#pragma unroll
    for (int k = 0; k < G; ++k) {
        const int a = (int)J.Q[k] + 1 - myN[k];   // eq. 1.1
        key |= (unsigned long long)((uint32_t)(a + 32768) & 0xFFFFu) << (16 * k);
    }
    if (sqf) {
        const unsigned peers = __match_any_sync(smask, key);
        if (lane == __ffs(peers) - 1) hist_insert(J, key, __popc(peers));
    }
}

// ---------------------------------------------------------------------
// kernels

template <int D>
__global__ void __launch_bounds__(256) k_plain(const KJob *__restrict__ jp)
{
    extern __shared__ __align__(16) uint8_t smem[];
    const KJob &J = *jp;
    stage_job(J, smem);
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    WarpStats st;
    for (uint64_t t = (uint64_t)blockIdx.x * nw + warp; t < J.n_tiles; t += (uint64_t)gridDim.x * nw)
        process_tile<D>(J, t, smem, lane, st);
    flush_stats(J, st, lane);
}

// Persistent: CTAs pull work items (a run of tiles of one job) from a counter
// until the queue is empty; a CTA restages tables only when its job changes.
template <int D>
__global__ void __launch_bounds__(256) k_persistent(const KJob *__restrict__ jobs,
                                                    const uint64_t *__restrict__ item_start,
                                                    uint32_t n_jobs, uint64_t n_items,
                                                    unsigned long long *counter, uint32_t item_tiles)
{
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ unsigned long long s_item;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int cur = -1;
    WarpStats st;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(counter, 1ull);
        __syncthreads();
        const uint64_t item = s_item;
        __syncthreads();   // everyone has read s_item
        if (item >= n_items) break;
        // job owning this item: item_start is ascending, item_start[n_jobs] = n_items
        uint32_t lo = 0, hi = n_jobs;
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (item_start[mid] <= item) lo = mid;
            else hi = mid;
        }
        const int jb = (int)lo;
        if (jb != cur) {
            if (cur >= 0) flush_stats(jobs[cur], st, lane);
            stage_job(jobs[jb], smem);
            __syncthreads();
            cur = jb;
        }
        const KJob &J = jobs[jb];
        const uint64_t t0 = (item - item_start[jb]) * item_tiles;
        const uint64_t t1 = min(t0 + item_tiles, J.n_tiles);
        for (uint64_t t = t0 + warp; t < t1; t += nw) process_tile<D>(J, t, smem, lane, st);
        __syncthreads();   // tables may be restaged next iteration
    }
    if (cur >= 0) flush_stats(jobs[cur], st, lane);
}

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

}  // namespace

// ---------------------------------------------------------------------
// host launch wrappers

using KernelFn = const void *;

static KernelFn plain_fn(int D)
{
    switch (D) {
    case 3: return (KernelFn)k_plain<3>;
    case 4: return (KernelFn)k_plain<4>;
    case 5: return (KernelFn)k_plain<5>;
    case 6: return (KernelFn)k_plain<6>;
    case 7: return (KernelFn)k_plain<7>;
    case 8: return (KernelFn)k_plain<8>;
    case 9: return (KernelFn)k_plain<9>;
    case 10: return (KernelFn)k_plain<10>;
    default: return nullptr;
    }
}

static KernelFn persistent_fn(int D)
{
    switch (D) {
    case 3: return (KernelFn)k_persistent<3>;
    case 4: return (KernelFn)k_persistent<4>;
    case 5: return (KernelFn)k_persistent<5>;
    case 6: return (KernelFn)k_persistent<6>;
    case 7: return (KernelFn)k_persistent<7>;
    case 8: return (KernelFn)k_persistent<8>;
    case 9: return (KernelFn)k_persistent<9>;
    case 10: return (KernelFn)k_persistent<10>;
    default: return nullptr;
    }
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
        for (KernelFn fn : {plain_fn(D), persistent_fn(D), fan_kernel(D, 1, false), fan_kernel(D, 1, true),
                            fan_kernel(D, 2, false), fan_kernel(D, 2, true)}) {
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

static KernelFn kernel_for(int D, uint32_t method, uint32_t words, bool persistent)
{
    if (method == 1) return fan_kernel(D, (int)words, persistent);
    return persistent ? persistent_fn(D) : plain_fn(D);
}

int max_ctas_per_sm(int D, uint32_t method, uint32_t words, int block, uint32_t smem_bytes,
                    bool persistent, int *out)
{
    int n = 0;
    KernelFn fn = kernel_for(D, method, words, persistent);
    if (!fn) return set_error(HWC_ERR_ARG, "degree %d has no kernel", D);
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

int launch_plain(const KJob *d_job, const KJob &h_job, const LaunchShape &sh, cudaStream_t s)
{
    int grid = sh.grid;
    if (grid <= 0) grid = device_sm_count();
    const uint64_t need = (h_job.n_tiles + (sh.block / 32) - 1) / (sh.block / 32);
    if ((uint64_t)grid > need) grid = (int)std::max<uint64_t>(need, 1);
    KernelFn fn = kernel_for((int)h_job.d, h_job.method, h_job.words, false);
    if (!fn) return set_error(HWC_ERR_ARG, "degree %u has no kernel", h_job.d);
    void *args[] = {(void *)&d_job};
    HWC_CUDA_TRY(cudaLaunchKernel(fn, dim3(grid), dim3(sh.block), args, h_job.smem_bytes, s));
    return HWC_OK;
}

int launch_persistent(int D, uint32_t method, uint32_t words, const KJob *d_jobs,
                      const uint64_t *d_item_start, uint32_t n_jobs, uint64_t n_items,
                      unsigned long long *d_counter, uint32_t max_smem, const LaunchShape &sh,
                      cudaStream_t s)
{
    KernelFn fn = kernel_for(D, method, words, true);
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
// Some callers cannot call cudaMalloc when they count: code that runs while a
// stream is being captured into a CUDA graph (allocation would break the
// capture), processes that reserve all device memory up front and hand out
// fixed pools, or host applications whose plug-in rules forbid device
// allocation.  This entry point keeps all of its working memory in one
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

template <int D>
__global__ void __launch_bounds__(256) k_na_count(const KJob J)
{
    extern __shared__ __align__(16) uint8_t smem[];
    stage_job(J, smem);
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    WarpStats st;
    for (uint64_t t = (uint64_t)blockIdx.x * nw + warp; t < J.n_tiles; t += (uint64_t)gridDim.x * nw)
        process_tile<D>(J, t, smem, lane, st);
    flush_stats(J, st, lane);
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

template <int D>
KernelFn na_count_fn()
{
    return (KernelFn)k_na_count<D>;
}

KernelFn na_count_kernel(int D)
{
    switch (D) {
    case 3: return na_count_fn<3>();
    case 4: return na_count_fn<4>();
    case 5: return na_count_fn<5>();
    case 6: return na_count_fn<6>();
    case 7: return na_count_fn<7>();
    case 8: return na_count_fn<8>();
    case 9: return na_count_fn<9>();
    case 10: return na_count_fn<10>();
    default: return nullptr;
    }
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
    if (fam->kind > HWC_FAM_MONIC_NOSUB_SAMPLED) return set_error(HWC_ERR_ARG, "unknown family kind");
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
    for (uint32_t k = 1; k <= g; ++k) {
        const hwc_tables_t *h = tables[k - 1];
        if (!h || !h->t || h->t->q != q || h->t->k != k)
            return set_error(HWC_ERR_ARG, "tables[%u] must be the tables of F_%u^%u", k - 1, q, k);
        const Tables *t = h->t;
        kj.Q[k - 1] = t->Q;
        kj.L[k - 1] = t->L;
        kj.barrett[k - 1] = (uint32_t)((1ull << 32) / t->L);
        kj.zech2[k - 1] = t->d_zech2;
        kj.zech3[k - 1] = t->d_zech3;
        kj.zech2w[k - 1] = t->d_zech2w;
        kj.coef_log[k - 1] = t->d_coef_log;
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
