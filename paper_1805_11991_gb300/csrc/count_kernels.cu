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
#include "hwc_internal.cuh"

#include <algorithm>

namespace hwc {
namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;

struct TabS {   // u16 table in shared memory
    const uint16_t *t;
    __device__ __forceinline__ uint32_t operator[](uint32_t u) const { return t[u]; }
};
struct TabG {   // u32 table in global memory (L1/L2 resident)
    const uint32_t *t;
    __device__ __forceinline__ uint32_t operator[](uint32_t u) const { return __ldg(t + u); }
};

__device__ __forceinline__ uint32_t addmod(uint32_t a, uint32_t b, uint32_t L)
{
    uint32_t s = a + b;
    return s >= L ? s - L : s;
}

// (g * j) mod L for g * j < 2^32, Barrett with bar = floor(2^32 / L)
__device__ __forceinline__ uint32_t mulmod_small(uint32_t g, uint32_t j, uint32_t L, uint32_t bar)
{
    uint32_t t = g * j;
    uint32_t qt = __umulhi(t, bar);
    uint32_t r = t - qt * L;
    return r >= L ? r - L : r;
}

__device__ __forceinline__ uint64_t mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// SplitMix64 output for state seed + (j+1)*gamma (Steele, Lea, Flood 2014)
__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t j)
{
    return mix64(seed + (j + 1) * 0x9E3779B97F4A7C15ull);
}

// ---------------------------------------------------------------------
// member decoding (Algorithm 1 line 3; family definitions in hwc.h)

template <int D>
__device__ __forceinline__ void decode_member(const KJob &J, uint64_t m, uint32_t (&c)[D + 1])
{
    uint64_t idx = J.first + m;
    uint32_t kind = J.kind;
    if (kind == HWC_FAM_MONIC_NOSUB_SAMPLED) {
        idx = __umul64hi(splitmix64_at(J.seed, idx), J.fam_mz);
        kind = HWC_FAM_MONIC_NOSUB;
    }
    const uint32_t q = J.q;
    const int ndig = (kind == HWC_FAM_ALL_DEG) ? D : D - 1;
    uint64_t r = idx;
#pragma unroll
    for (int i = 0; i <= D; ++i) {
        if (i < ndig) {
            if (r >> 32) {
                c[i] = (uint32_t)(r % q);
                r /= q;
            } else {
                uint32_t r32 = (uint32_t)r;
                c[i] = r32 % q;
                r = r32 / q;
            }
        }
    }
    if (kind == HWC_FAM_ALL_DEG) {
        c[D] = 1 + (uint32_t)r;
    } else {
        c[D - 1] = 0;
        c[D] = 1;
    }
}

// ---------------------------------------------------------------------
// square-freeness: gcd(f, f') in Zech arithmetic over F_q (k = 1 tables).
// Elements as logs, zero = L1.

template <class Tab>
struct FqLog {
    Tab T;
    uint32_t L;
    __device__ __forceinline__ uint32_t mul(uint32_t a, uint32_t b) const
    {
        return (a == L || b == L) ? L : addmod(a, b, L);
    }
    __device__ __forceinline__ uint32_t neg(uint32_t a) const
    {
        return a == L ? L : addmod(a, L >> 1, L);
    }
    __device__ __forceinline__ uint32_t add(uint32_t a, uint32_t b) const
    {
        if (a == L) return b;
        if (b == L) return a;
        uint32_t n = addmod(a, L - b, L);
        uint32_t z = T[n];
        return z >= 2 * L ? L : addmod(b, z, L);
    }
};

template <int D, class Tab>
__device__ bool squarefree(const FqLog<Tab> &F, const uint32_t *coef1, uint32_t p,
                           const uint32_t (&c)[D + 1])
{
    const uint32_t Z = F.L;
    uint32_t P[2][D + 1];
    int dg[2];
    for (int i = 0; i <= D; ++i) P[0][i] = coef1[c[i]];
    // f' = sum i c_i x^(i-1); the integer i is the F_p digit (i mod p)
    for (int i = 1; i <= D; ++i) P[1][i - 1] = F.mul(coef1[i % p], P[0][i]);
    P[1][D] = Z;
    dg[0] = D;
    dg[1] = D - 1;
    while (dg[0] >= 0 && P[0][dg[0]] == Z) --dg[0];
    while (dg[1] >= 0 && P[1][dg[1]] == Z) --dg[1];
    if (dg[1] < 0) return false;
    int a = 0, b = 1;
    while (dg[b] >= 0) {
        const int db = dg[b];
        const uint32_t il = (F.L - P[b][db]) % F.L;   // inverse of the lead
        for (int t = dg[a]; t >= db; --t) {
            if (P[a][t] == Z) continue;
            const uint32_t cf = F.mul(P[a][t], il);
            for (int i = 0; i <= db; ++i)
                P[a][t - db + i] = F.add(P[a][t - db + i], F.neg(F.mul(cf, P[b][i])));
        }
        int da = db - 1;
        while (da >= 0 && P[a][da] == Z) --da;
        dg[a] = da;
        int tmp = a; a = b; b = tmp;
    }
    return dg[a] == 0;
}

// ---------------------------------------------------------------------
// one field: sum over x in F_Q^x of chi(f(x)) for this lane's share of x

template <int D, class Tab>
__device__ __noinline__ int slow_chi(const Tab T, uint32_t L, const uint32_t (&lam)[D + 1],
                                     uint32_t nz, uint32_t j)
{
    uint32_t l = lam[D];
    bool zero = false;
#pragma unroll
    for (int i = D - 1; i >= 0; --i) {
        if (!zero) l = addmod(l, j, L);
        if ((nz >> i) & 1u) {
            if (zero) {
                l = lam[i];
                zero = false;
            } else {
                uint32_t n = addmod(l, L - lam[i], L);
                uint32_t z = T[n];
                if (z >= 2 * L) zero = true;
                else l = addmod(lam[i], z, L);
            }
        }
    }
    return zero ? 0 : ((l & 1u) ? -1 : 1);
}

template <int D, class Tab>
__device__ __forceinline__ int field_chi_sum(const Tab T, uint32_t L, uint32_t bar,
                                             const uint32_t (&lam)[D + 1], uint32_t nz, int lane)
{
    const uint32_t L2 = 2 * L;
    int S = 0;
    if (nz == 0) {   // f = c_D x^D
        for (uint32_t j = lane; j < L; j += 32) S += ((lam[D] + (uint32_t)D * j) & 1u) ? -1 : 1;
        return S;
    }
    const int i1 = 31 - __clz(nz);
    const int is = __ffs(nz) - 1;
    const uint32_t g1 = (uint32_t)(D - i1);
    const uint32_t negl1 = L - lam[i1];
    const uint32_t lamlast = lam[is];
    for (uint32_t j0 = 0; j0 < L; j0 += 64) {
        uint32_t jA = j0 + lane, jB = j0 + 32 + lane;
        const bool vA = jA < L, vB = jB < L;
        jA = vA ? jA : 0;
        jB = vB ? jB : 0;
        uint32_t uA = addmod(lam[D], mulmod_small(g1, jA, L, bar), L) + negl1;
        uint32_t uB = addmod(lam[D], mulmod_small(g1, jB, L, bar), L) + negl1;
        uint32_t lp = lam[i1];
        int ip = i1;
#pragma unroll
        for (int i = D - 2; i >= 0; --i) {
            if (i >= i1 || !((nz >> i) & 1u)) continue;
            const uint32_t dl = addmod(lp, L - lam[i], L);
            const uint32_t gap = (uint32_t)(ip - i);
            uint32_t eA, eB;
            if (gap == 1) {
                eA = addmod(dl, jA, L);
                eB = addmod(dl, jB, L);
            } else {
                eA = addmod(dl, mulmod_small(gap, jA, L, bar), L);
                eB = addmod(dl, mulmod_small(gap, jB, L, bar), L);
            }
            const uint32_t zA = T[uA], zB = T[uB];
            uA = min(zA + eA, L2);
            uB = min(zB + eB, L2);
            lp = lam[i];
            ip = i;
        }
        const uint32_t zA = T[uA], zB = T[uB];
        const uint32_t tailA = (uint32_t)is * jA, tailB = (uint32_t)is * jB;
        int cA = ((lamlast + zA + tailA) & 1u) ? -1 : 1;
        int cB = ((lamlast + zB + tailB) & 1u) ? -1 : 1;
        const bool pA = vA && zA >= L2, pB = vB && zB >= L2;
        if (__any_sync(kFull, pA || pB)) {
            if (pA) cA = slow_chi<D>(T, L, lam, nz, jA);
            if (pB) cB = slow_chi<D>(T, L, lam, nz, jB);
        }
        S += (vA ? cA : 0) + (vB ? cB : 0);
    }
    return S;
}

// ---------------------------------------------------------------------
// histogram

__device__ __forceinline__ void hist_insert(const KJob &J, unsigned long long key, uint32_t cnt)
{
    uint32_t h = (uint32_t)mix64(key) & J.hmask;
    for (uint32_t probe = 0; probe <= J.hmask; ++probe) {
        unsigned long long cur = *((volatile unsigned long long *)&J.hkeys[h]);
        if (cur == kEmptyKey) cur = atomicCAS(&J.hkeys[h], kEmptyKey, key);
        if (cur == kEmptyKey || cur == key) {
            atomicAdd(&J.hcounts[h], (unsigned long long)cnt);
            return;
        }
        h = (h + 1) & J.hmask;
    }
    atomicOr(&J.stats[2], 1ull);   // table full
}

struct WarpStats {
    uint32_t examined = 0, sqf = 0;
};

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
        if (J.tab_off[0] != kWideTable) {
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
            if (J.tab_off[k] != kWideTable)
                S = field_chi_sum<D>(TabS{s16 + J.tab_off[k]}, L, J.barrett[k], lam, nz, lane);
            else
                S = field_chi_sum<D>(TabG{J.zech2w[k]}, L, J.barrett[k], lam, nz, lane);
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

__device__ void process_tile_any(const KJob &J, uint64_t tile, const uint8_t *smem, int lane,
                                 WarpStats &st)
{
    switch (J.d) {
    case 3: process_tile<3>(J, tile, smem, lane, st); break;
    case 4: process_tile<4>(J, tile, smem, lane, st); break;
    case 5: process_tile<5>(J, tile, smem, lane, st); break;
    case 6: process_tile<6>(J, tile, smem, lane, st); break;
    case 7: process_tile<7>(J, tile, smem, lane, st); break;
    case 8: process_tile<8>(J, tile, smem, lane, st); break;
    case 9: process_tile<9>(J, tile, smem, lane, st); break;
    case 10: process_tile<10>(J, tile, smem, lane, st); break;
    default: break;
    }
}

// copy the job's tables into shared memory (all threads of the CTA)
__device__ void stage_job(const KJob &J, uint8_t *smem)
{
    uint16_t *s16 = reinterpret_cast<uint16_t *>(smem);
    uint32_t *s32 = reinterpret_cast<uint32_t *>(smem);
    for (uint32_t k = 0; k < J.g; ++k) {
        if (J.tab_off[k] != kWideTable) {
            const uint32_t n = 2 * J.L[k] + 1;
            const uint16_t *src = J.zech2[k];
            uint16_t *dst = s16 + J.tab_off[k];
            for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
        }
        const uint32_t *src = J.coef_log[k];
        uint32_t *dst = s32 + J.coef_off[k];
        for (uint32_t i = threadIdx.x; i < J.q; i += blockDim.x) dst[i] = src[i];
    }
}

__device__ __forceinline__ void flush_stats(const KJob &J, WarpStats &st, int lane)
{
    if (lane == 0 && (st.examined | st.sqf)) {
        atomicAdd(&J.stats[0], (unsigned long long)st.examined);
        atomicAdd(&J.stats[1], (unsigned long long)st.sqf);
    }
    st.examined = st.sqf = 0;
}

// ---------------------------------------------------------------------
// kernels

__global__ void k_plain(const KJob *__restrict__ jp)
{
    extern __shared__ __align__(16) uint8_t smem[];
    const KJob &J = *jp;
    stage_job(J, smem);
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    WarpStats st;
    for (uint64_t t = (uint64_t)blockIdx.x * nw + warp; t < J.n_tiles; t += (uint64_t)gridDim.x * nw)
        process_tile_any(J, t, smem, lane, st);
    flush_stats(J, st, lane);
}

__global__ void k_persistent(const KJob *__restrict__ jobs, const uint64_t *__restrict__ item_start,
                             uint32_t n_jobs, uint64_t n_items, unsigned long long *counter,
                             uint32_t item_tiles)
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
            uint32_t mid = (lo + hi) >> 1;
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
        for (uint64_t t = t0 + warp; t < t1; t += nw) process_tile_any(J, t, smem, lane, st);
        __syncthreads();   // tables may be restaged next iteration
    }
    if (cur >= 0) flush_stats(jobs[cur], st, lane);
}

__global__ void k_clear(const KJob *__restrict__ jobs, uint32_t n_jobs, unsigned long long *counter)
{
    const uint32_t jb = blockIdx.y;
    if (jb == 0 && blockIdx.x == 0 && threadIdx.x == 0 && counter) *counter = 0;
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

int prepare_count_kernels(void)
{
    static std::mutex mu;
    static bool done[64] = {};
    int dev = 0;
    HWC_CUDA_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(mu);
    if (dev >= 0 && dev < 64 && done[dev]) return HWC_OK;
    const int optin = (int)device_smem_optin();
    HWC_CUDA_TRY(cudaFuncSetAttribute((const void *)k_plain, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
    HWC_CUDA_TRY(cudaFuncSetAttribute((const void *)k_persistent, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
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

int max_ctas_per_sm(int block, uint32_t smem_bytes, bool persistent, int *out)
{
    int n = 0;
    const void *fn = persistent ? (const void *)k_persistent : (const void *)k_plain;
    HWC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, block, smem_bytes));
    *out = n;
    return HWC_OK;
}

int launch_clear(const KJob *d_jobs, uint32_t n_jobs, unsigned long long *d_counter, cudaStream_t s)
{
    dim3 grid(device_sm_count(), std::max<uint32_t>(n_jobs, 1));
    k_clear<<<grid, 256, 0, s>>>(d_jobs, n_jobs, d_counter);
    HWC_CUDA_TRY(cudaGetLastError());
    return HWC_OK;
}

int launch_plain(const KJob *d_job, const KJob &h_job, const LaunchShape &sh, cudaStream_t s)
{
    int grid = sh.grid;
    if (grid <= 0) grid = device_sm_count();
    uint64_t need = (h_job.n_tiles + (sh.block / 32) - 1) / (sh.block / 32);
    if ((uint64_t)grid > need) grid = (int)std::max<uint64_t>(need, 1);
    k_plain<<<grid, sh.block, h_job.smem_bytes, s>>>(d_job);
    HWC_CUDA_TRY(cudaGetLastError());
    return HWC_OK;
}

int launch_persistent(const KJob *d_jobs, const uint64_t *d_item_start, uint32_t n_jobs,
                      uint64_t n_items, unsigned long long *d_counter, uint32_t max_smem,
                      const LaunchShape &sh, cudaStream_t s)
{
    k_persistent<<<sh.grid, sh.block, max_smem, s>>>(d_jobs, d_item_start, n_jobs, n_items, d_counter,
                                                    (uint32_t)sh.item_tiles);
    HWC_CUDA_TRY(cudaGetLastError());
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
