// horner.cuh -- per-member Horner count kernel (sm_103a); instantiated per
// degree in horner_a.cu (d = 3..6) and horner_b.cu (d = 7..10).
//
// One warp handles a tile of 32 consecutive members of a family:
//   1. each lane decodes one member index into coefficient digits (the choice
//      of f in Algorithm 1) and tests it for square-freeness by Euclid's
//      algorithm on gcd(f, f') in Zech arithmetic over F_q;
//   2. for every square-free member of the tile (uniform loop) and every
//      k = 1..g the 32 lanes sweep x = alpha^j over F_Q^x (the evaluation
//      loop of Algorithm 1), two
//      x per lane per step, evaluating f by Horner's rule in the log domain
//      with one Zech lookup per nonzero coefficient (eq. 2.1, 3.1-3.2), and
//      sum chi(f(x)) = (-1)^log (the parity of the log, L being even);
//   3. #C_k = Q + sum_x chi(f(x)) + 1 + chi(f(inf)) (Sec. 1.1), i.e.
//      r^0 + 2 r^sq + 1 + chi(f(inf)); the lanes' tuples are aggregated
//      within the warp (match.any) and added into an open-addressing hash
//      in global memory (the histogram increment of Algorithm 1, weight 1).
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
#pragma once
#include "count_common.cuh"

#include <algorithm>

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

// sum of chi(f(x)) over this lane's share of the field's points x = alpha^j:
// j = pts[i] for i < npts (one point per Frobenius orbit), or every j < L when
// pts is null; zeros += the points with f(x) = 0
template <int D, bool TRIPLE, class Tab>
__device__ __forceinline__ int field_chi_sum(const Tab T, uint32_t L, uint32_t bar,
                                             const uint32_t (&lam)[D + 1], uint32_t nz, int lane,
                                             const uint32_t *__restrict__ pts, uint32_t npts, int &zeros)
{
    const uint32_t cap = TRIPLE ? 3 * L : 2 * L;
    int S = 0;
    if (nz == 0) {   // f = c_D x^D (never 0 at x != 0)
        for (uint32_t i = lane; i < npts; i += 32) {
            const uint32_t j = pts ? __ldg(pts + i) : i;
            S += ((lam[D] + (uint32_t)D * j) & 1u) ? -1 : 1;
        }
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
    for (uint32_t i0 = 0; i0 < npts; i0 += 64) {
        const uint32_t iA = i0 + lane, iB = i0 + 32 + lane;
        const bool vA = iA < npts, vB = iB < npts;
        uint32_t xA = vA ? iA : 0, xB = vB ? iB : 0;
        if (pts) {
            xA = __ldg(pts + xA);
            xB = __ldg(pts + xB);
        }
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
            zeros += (pA && cA == 0) + (pB && cB == 0);
        }
        S += (vA ? cA : 0) + (vB ? cB : 0);
    }
    return S;
}

// ---------------------------------------------------------------------
// one tile of 32 members, processed by one warp

template <int D>
__device__ __forceinline__ void process_tile(const KJob &J, uint64_t tile, const uint8_t *smem, int lane,
                             WarpStats &st)
{
    constexpr int G = (D - 1) / 2;
    const uint64_t m = tile * kTileMembers + lane;
    const bool valid = m < J.count;
    uint32_t c[D + 1];
#pragma unroll
    for (int i = 0; i <= D; ++i) c[i] = 0;
    c[D] = 1;
    // reduced families: weight mult(f) of the member's pattern, counted for f
    // and for its quadratic twist
    const bool reduced = J.kind == HWC_FAM_REDUCED;
    unsigned long long wgt = 1;
    if (valid) {
        if (reduced) wgt = J.red_mult[decode_reduced<D>(J, J.first + m, c)];
        else decode_member<D>(J, m, c);
    }

    const uint16_t *s16 = reinterpret_cast<const uint16_t *>(smem);
    const uint32_t *s32 = reinterpret_cast<const uint32_t *>(smem);

    bool sqf = false;
    if (valid) {
        const uint32_t *coef1 = s32 + J.coef_off[0];
        if (J.tab_kind[0] == kTab17Smem) {
            FqLog<Tab17> F{Tab17{s16 + J.tab_off[0], reinterpret_cast<const uint32_t *>(s16 + J.tab_hi_off[0]),
                                 J.L[0]},
                           J.L[0]};
            sqf = squarefree<D>(F, coef1, J.p, c);
        } else if (J.tab_kind[0] != kTabDoubleGlobal) {
            FqLog<TabS> F{TabS{s16 + J.tab_off[0]}, J.L[0]};
            sqf = squarefree<D>(F, coef1, J.p, c);
        } else {
            FqLog<TabG> F{TabG{J.zech2w[0]}, J.L[0]};
            sqf = squarefree<D>(F, coef1, J.p, c);
        }
    }
    const unsigned vmask = __ballot_sync(kFull, valid);
    const unsigned smask = __ballot_sync(kFull, sqf);
    if (reduced) {   // weighted square-free count: 2 mult(f) per member (f and its twist)
        unsigned long long ws = sqf ? 2 * wgt : 0ull;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) ws += __shfl_xor_sync(kFull, ws, o);
        if (lane == 0) {
            st.examined += __popc(vmask);
            st.sqf += ws;
        }
    } else if (lane == 0) {
        st.examined += __popc(vmask);
        st.sqf += __popc(smask);
    }
    unsigned todo = J.unfiltered ? vmask : smask;

    int myE[G], myZ[G];   // per field m = k+1: sum of chi and zeros over its points (x = 0 in field 1)
#pragma unroll
    for (int k = 0; k < G; ++k) myE[k] = myZ[k] = 0;

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
            int S, Zr = 0;
            const uint32_t kind = J.tab_kind[k];
            const uint32_t *pts = J.reps[k];
            const uint32_t np = J.npts[k];
            if (kind == kTabTripleSmem)
                S = field_chi_sum<D, true>(TabS{s16 + J.tab_off[k]}, L, J.barrett[k], lam, nz, lane, pts, np, Zr);
            else if (kind == kTabDoubleSmem)
                S = field_chi_sum<D, false>(TabS{s16 + J.tab_off[k]}, L, J.barrett[k], lam, nz, lane, pts, np, Zr);
            else if (kind == kTab17Smem)
                S = field_chi_sum<D, false>(
                    Tab17{s16 + J.tab_off[k], reinterpret_cast<const uint32_t *>(s16 + J.tab_hi_off[k]), L}, L,
                    J.barrett[k], lam, nz, lane, pts, np, Zr);
            else
                S = field_chi_sum<D, false>(TabG{J.zech2w[k]}, L, J.barrett[k], lam, nz, lane, pts, np, Zr);
            if (lane == 0 && !pts) {   // x = 0 (in F_q; in every field when every point is evaluated)
                if (cc[0] != 0) S += (lam[0] & 1u) ? -1 : 1;
                else Zr += 1;
            }
            S = __reduce_add_sync(kFull, S);
            Zr = __reduce_add_sync(kFull, Zr);
            if (lane == src) {
                myE[k] = S;
                myZ[k] = Zr;
            }
        }
    }
    // #C_k = Q_k + S_k + 1 + chi(c_{2g+2})  (points at infinity; chi of c_d in F_{q^k})
    int32_t myN[G];
    {
        int Sk[G];
        orbit_combine<G>(J, myE, myZ, Sk);
#pragma unroll
        for (int k = 0; k < G; ++k) {
            int inf = 1;
            if (D == 2 * G + 2) inf += (s32[J.coef_off[k] + c[D]] & 1u) ? -1 : 1;
            myN[k] = (int32_t)J.Q[k] + Sk[k] + inf;
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
    unsigned long long key = 0, tkey = 0;   // tkey: the quadratic twist, a_k -> (-1)^k a_k
    if (J.lam_mode) {
        // (a_1..a_g, lambda(f)) of eq. 1.2: the orbit zeros of exact degree m are
        // the irreducible factors of degree m; what is left is one factor, or two
        // of degree g+1 when chi(disc f) = +1 (Stickelberger)
        uint32_t used = 0;
        unsigned long long lam = 0;
#pragma unroll
        for (int m = 1; m <= G; ++m) {
            const uint32_t nm = (uint32_t)myZ[m - 1];
            lam |= (unsigned long long)(nm & 0xFu) << (4 * (m - 1));
            used += (uint32_t)m * nm;
        }
        if (sqf && D == 2 * G + 2 && used == 0) {
            int dc;
            const uint32_t *coef1 = s32 + J.coef_off[0];
            if (J.tab_kind[0] == kTab17Smem)
                dc = disc_chi<D>(FqLog<Tab17>{Tab17{s16 + J.tab_off[0],
                                                    reinterpret_cast<const uint32_t *>(s16 + J.tab_hi_off[0]), J.L[0]},
                                              J.L[0]},
                                 coef1, J.p, J.q, c);
            else if (J.tab_kind[0] != kTabDoubleGlobal)
                dc = disc_chi<D>(FqLog<TabS>{TabS{s16 + J.tab_off[0]}, J.L[0]}, coef1, J.p, J.q, c);
            else
                dc = disc_chi<D>(FqLog<TabG>{TabG{J.zech2w[0]}, J.L[0]}, coef1, J.p, J.q, c);
            if (dc > 0) lam |= 1ull << (4 * G);
        }
#pragma unroll
        for (int k = 0; k < G; ++k) {
            const int a = (int)J.Q[k] + 1 - myN[k];   // eq. 1.1
            const int at = (k & 1) ? a : -a;
            key |= (unsigned long long)(uint32_t)(a + J.key_bias[k]) << J.key_shift[k];
            tkey |= (unsigned long long)(uint32_t)(at + J.key_bias[k]) << J.key_shift[k];
        }
        key |= lam << J.lam_shift;
        tkey |= lam << J.lam_shift;
    } else {
#pragma unroll
        for (int k = 0; k < G; ++k) {
            const int a = (int)J.Q[k] + 1 - myN[k];   // eq. 1.1
            const int at = (k & 1) ? a : -a;
            key |= (unsigned long long)((uint32_t)(a + 32768) & 0xFFFFu) << (16 * k);
            tkey |= (unsigned long long)((uint32_t)(at + 32768) & 0xFFFFu) << (16 * k);
        }
    }
    if (reduced) {
        if (sqf) {
            hist_insert(J, key, wgt);
            hist_insert(J, tkey, wgt);
        }
        return;
    }
    if (sqf) {
        const unsigned peers = __match_any_sync(smask, key);
        if (lane == __ffs(peers) - 1) hist_insert(J, key, __popc(peers));
    }
}

// ---------------------------------------------------------------------
// kernels

// Persistent: CTAs pull work items (a run of tiles of one job) from a counter
// until the queue is empty; a CTA restages tables only when its job changes.
template <int D>
__device__ __forceinline__ void persistent_body(const KJob *__restrict__ jobs, const uint64_t *__restrict__ item_start,
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

// up to 256 threads (several CTAs per SM)
template <int D>
__global__ void __launch_bounds__(256) k_persistent(const KJob *__restrict__ jobs,
                                                    const uint64_t *__restrict__ item_start, uint32_t n_jobs,
                                                    uint64_t n_items, unsigned long long *counter,
                                                    uint32_t item_tiles)
{
    persistent_body<D>(jobs, item_start, n_jobs, n_items, counter, item_tiles);
}

// up to 768 threads (512 for degrees >= 7, whose longer chains need more than
// 80 registers): for jobs whose tables leave room for one CTA per SM (the
// 17-bit Zech table of F_{293^2}, the u16 table of F_{13^4}), which then still
// keep 16-24 warps resident
template <int D>
__global__ void __launch_bounds__(D <= 6 ? 768 : 512, 1) k_persistent_wide(const KJob *__restrict__ jobs,
                                                            const uint64_t *__restrict__ item_start,
                                                            uint32_t n_jobs, uint64_t n_items,
                                                            unsigned long long *counter, uint32_t item_tiles)
{
    persistent_body<D>(jobs, item_start, n_jobs, n_items, counter, item_tiles);
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

template <int D>
const void *horner_pick(int which)
{
    if (which == 1) return (const void *)k_persistent<D>;
    if (which == 3) return (const void *)k_persistent_wide<D>;
    if (which == 0) return nullptr;   // plain runs use the persistent kernel, one job per launch
    return (const void *)k_na_count<D>;
}

}  // namespace
}  // namespace hwc
