// classes.cuh -- class-sharing count kernel for sampled families drawn with
// many members per class; instantiated for degrees 3..6 in cls_a.cu.
//
// A sampled member f = u + c_1 x + c_0 of the monic family with c_{d-1} = 0
// shares u(x) = x^d + c_{d-2} x^(d-2) + ... + c_2 x^2 with every member whose
// high digits (c_2..c_{d-2}, the "class") agree.  Before the count kernel the
// samples are sorted by class on the device (a counting sort: count per
// class, one scan that also writes the tile list, a scatter of the low digits
// c_0 + c_1 q).  A warp then takes a tile of up to 32 samples of one class,
// one sample per lane.  For each batch of 64 points x = alpha^j the lanes
// evaluate log u(x) by the Zech-index chain (two points each) and stage
// (log u, log x) in the warp's shared scratch; then every lane walks the 64
// staged points for its own member with two Zech additions (eq. 2.1):
//     y = u + c_1 x = c_1 x (1 + u / (c_1 x)),   f(x) = y + c_0 = c_0 (1 + y / c_0),
// and the quadratic character of f(x) is the parity of its log (Sec. 3.1).
// A vanishing partial sum (u = 0, y = 0 or f = 0: the poison of the Zech
// table) sends that lane and point to a branchy step that also counts the
// zeros.  Per member and point this is two table reads instead of one per
// nonzero coefficient; the chain for u is shared by the tile's members.
// Counts, orbit recombination and the histogram follow the per-member kernel
// (horner.cuh): #C_k = Q + sum_x chi(f(x)) + 1 + chi(f(inf)) (Sec. 1.1).
#pragma once
#include "fanout.cuh"

namespace hwc {
namespace {

// sum of chi and zeros of the lane's member f = u + c_1 x + c_0 over the
// staged points [0, nb); l1 / l0 = log c_1 / log c_0, z1 / z0: c_1 / c_0 = 0
template <class Tab>
__device__ __forceinline__ void cls_points(const Tab T, uint32_t L, const uint2 *st, uint32_t nb, uint32_t l1,
                                           uint32_t l0, bool z1, bool z0, int &odd, int &zeros)
{
    const uint32_t cap = 2 * L;
#pragma unroll 4
    for (uint32_t p = 0; p < nb; ++p) {
        const uint2 ux = st[p];
        const uint32_t U = ux.x, X = ux.y;
        uint32_t lcx = l1 + X;
        lcx = min(lcx, lcx - L);                       // log(c_1 x) in [0, L)
        const uint32_t i1 = U + L - lcx;               // in (0, 2L]: u = 0 (U = L) and lcx = 0 read the poison at 2L
        const uint32_t t1 = lcx + T[i1];
        uint32_t ly = min(t1, t1 - L);                 // log y; >= L when y = 0 or u = 0
        ly = z1 ? U : ly;                              // c_1 = 0: y = u
        const uint32_t i2 = min(ly + L - l0, cap);
        const uint32_t w2 = T[i2];
        const uint32_t lf = z0 ? ly : l0 + w2;         // parity of log f
        const bool rare = U >= L || ly >= L || (!z0 && w2 >= cap);
        odd += rare ? 0 : (int)(lf & 1u);
        if (rare) {   // explicit zeros: u = 0, y = 0 or f = 0
            bool yz;
            uint32_t lyy;
            if (U >= L) {
                yz = z1;
                lyy = lcx;
            } else if (z1) {
                yz = false;
                lyy = U;
            } else {
                const uint32_t w = T[U + L - lcx];
                yz = w >= cap;
                const uint32_t t = lcx + w;
                lyy = min(t, t - L);
            }
            if (yz) {
                if (z0) ++zeros;
                else odd += (int)(l0 & 1u);
            } else if (z0) {
                odd += (int)(lyy & 1u);
            } else {
                const uint32_t w = T[lyy + L - l0];
                if (w >= cap) ++zeros;
                else odd += (int)((l0 + w) & 1u);
            }
        }
    }
}

// one field: E = sum of chi(f(x)), Z = zeros over the field's points
// (J.reps[k], or every x = alpha^j, j < L), for the lane's member
template <int D, class Tab>
__device__ __forceinline__ void cls_field(const KJob &J, int k, const Tab T, const uint32_t (&lam)[D + 1], uint32_t nz,
                                          uint2 *st, int lane, bool active, int &E, int &Z)
{
    const uint32_t L = J.L[k];
    const uint32_t bar = J.barrett[k];
    HChain<D> H;
    make_hchain<D, 2>(H, lam, nz, L);
    const uint32_t *__restrict__ pts = J.reps[k];
    const uint32_t np = J.npts[k];
    const bool z1 = !((nz >> 1) & 1u), z0 = !(nz & 1u);
    int odd = 0, zeros = 0;
    for (uint32_t j0 = 0; j0 < np; j0 += 64) {
        const uint32_t iA = j0 + lane, iB = j0 + 32 + lane;
        uint32_t xA = iA < np ? iA : 0, xB = iB < np ? iB : 0;
        if (pts) {
            xA = __ldg(pts + min(iA, np - 1));
            xB = __ldg(pts + min(iB, np - 1));
        }
        uint32_t uA, uB;
        log_y_pair<D, false, Tab, 2>(T, L, bar, H, lam, nz, xA, xB, uA, uB);
        st[lane] = make_uint2(uA, xA);
        st[32 + lane] = make_uint2(uB, xB);
        __syncwarp();
        if (active) cls_points(T, L, st, min(64u, np - j0), lam[1], lam[0], z1, z0, odd, zeros);
        __syncwarp();   // the next batch rewrites the staged points
    }
    E = (int)np - zeros - 2 * odd;
    Z = zeros;
}

// one tile: up to 32 sorted samples of one class
template <int D>
__device__ __forceinline__ void process_class_tile(const KJob &J, uint64_t tile, const uint8_t *smem, uint2 *st,
                                                   int lane, WarpStats &st_)
{
    constexpr int G = (D - 1) / 2;
    const uint2 tl = J.cls_tiles[tile];
    if (tl.x == 0xFFFFFFFFu) return;   // past the last tile of the sort
    const uint32_t cls = tl.x, start = tl.y;
    const uint32_t n = min(32u, J.cls_cnt[cls] - start);   // cls_cnt: end of the class after the scatter
    const bool valid = (uint32_t)lane < n;
    const uint32_t q = J.q;
    const uint32_t mi = valid ? J.cls_sorted[start + lane] : 0u;
    uint32_t c[D + 1];
    c[0] = mi % q;
    c[1] = mi / q;
    {
        uint32_t r = cls;
#pragma unroll
        for (int i = 2; i <= D - 2; ++i) {
            c[i] = r % q;
            r /= q;
        }
    }
    c[D - 1] = 0;
    c[D] = 1;

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
    if (lane == 0) {
        st_.examined += __popc(vmask);
        st_.sqf += __popc(smask);
    }
    if (smask == 0) return;
    uint32_t nz = 0;
#pragma unroll
    for (int i = 0; i < D; ++i) nz |= (c[i] != 0 ? 1u : 0u) << i;
    // the class digits are the same in every lane: the chain's positions 2..D
    // agree across the warp; positions 0, 1 are the lane's own

    int myE[G], myZ[G];
#pragma unroll
    for (int k = 0; k < G; ++k) {
        const uint32_t *coefk = s32 + J.coef_off[k];
        uint32_t lam[D + 1];
#pragma unroll
        for (int i = 0; i <= D; ++i) lam[i] = coefk[c[i]];
        int E = 0, Z = 0;
        const uint32_t kind = J.tab_kind[k];
        if (kind == kTab17Smem)
            cls_field<D>(J, k, Tab17{s16 + J.tab_off[k], reinterpret_cast<const uint32_t *>(s16 + J.tab_hi_off[k]), J.L[k]},
                         lam, nz, st, lane, sqf, E, Z);
        else if (kind == kTabDoubleSmem)
            cls_field<D>(J, k, TabS{s16 + J.tab_off[k]}, lam, nz, st, lane, sqf, E, Z);
        else
            cls_field<D>(J, k, TabG{J.zech2w[k]}, lam, nz, st, lane, sqf, E, Z);
        if (!J.reps[k]) {   // x = 0 (in F_q; in every field when every point is evaluated)
            if (c[0] != 0) E += (lam[0] & 1u) ? -1 : 1;
            else Z += 1;
        }
        myE[k] = E;
        myZ[k] = Z;
    }
    int Sk[G];
    orbit_combine<G>(J, myE, myZ, Sk);
    unsigned long long key = 0;
#pragma unroll
    for (int k = 0; k < G; ++k) {
        int inf = 1;
        if (D == 2 * G + 2) inf += (s32[J.coef_off[k] + c[D]] & 1u) ? -1 : 1;
        const int N = (int)J.Q[k] + Sk[k] + inf;
        const int a = (int)J.Q[k] + 1 - N;   // eq. 1.1
        key |= (unsigned long long)((uint32_t)(a + 32768) & 0xFFFFu) << (16 * k);
    }
    if (sqf) {
        const unsigned peers = __match_any_sync(smask, key);
        if (lane == __ffs(peers) - 1) hist_insert(J, key, __popc(peers));
    }
}

template <int D>
__device__ __forceinline__ void cls_body(const KJob *__restrict__ jobs, const uint64_t *__restrict__ item_start,
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
        __syncthreads();
        if (item >= n_items) break;
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
        uint2 *wst = reinterpret_cast<uint2 *>(smem + J.warp_off + warp * kClsWarpBytes);
        const uint64_t t0 = (item - item_start[jb]) * item_tiles;
        const uint64_t t1 = min(t0 + item_tiles, J.n_tiles);
        for (uint64_t t = t0 + warp; t < t1; t += nw) process_class_tile<D>(J, t, smem, wst, lane, st);
        __syncthreads();
    }
    if (cur >= 0) flush_stats(jobs[cur], st, lane);
}

template <int D>
__global__ void __launch_bounds__(256) k_cls_persistent(const KJob *__restrict__ jobs,
                                                        const uint64_t *__restrict__ item_start, uint32_t n_jobs,
                                                        uint64_t n_items, unsigned long long *counter,
                                                        uint32_t item_tiles)
{
    cls_body<D>(jobs, item_start, n_jobs, n_items, counter, item_tiles);
}

// one CTA per SM of up to 768 threads: for tables that fill shared memory
// (the 17-bit Zech table of F_{293^2})
template <int D>
__global__ void __launch_bounds__(768, 1) k_cls_persistent_wide(const KJob *__restrict__ jobs,
                                                                const uint64_t *__restrict__ item_start,
                                                                uint32_t n_jobs, uint64_t n_items,
                                                                unsigned long long *counter, uint32_t item_tiles)
{
    cls_body<D>(jobs, item_start, n_jobs, n_items, counter, item_tiles);
}

template <int D>
const void *cls_pick(int which)
{
    return which == 3 ? (const void *)k_cls_persistent_wide<D> : (const void *)k_cls_persistent<D>;
}

}  // namespace
}  // namespace hwc
