// fanout.cuh -- c_0 fan-out count kernel for enumerated families; instantiated
// per degree in fanout_a.cu .. fanout_e.cu.
//
// Consecutive members of a family differ first in c_0 (digit 0 of the member
// index), so q consecutive members f_c = g + c (c in F_q) share
// g(x) = f(x) - c_0 = x h(x), h(x) = c_d x^(d-1) + ... + c_1.  One warp takes
// such a group.  For every x = alpha^j in F_Q^x the lanes evaluate h(x) by the
// Zech-index Horner chain (eq. 2.1; one table read per nonzero c_i, i >= 1),
// form log y = log h(x) + j, and then do the last Zech addition y + c and the
// quadratic character for all q members at once: row y of the fan-out table
// holds the q bits [chi(y + c) = -1].  The rows of the lane's x are summed
// position by position with bit-sliced carry-save counters (8 inputs per
// block), and the warp adds its lanes' counters with a shuffle butterfly.
// With n_0 = #{x : y = 0} (x = 0 included), cnt_c the row-bit counts and z_c
// the number of x with y = -c != 0 (rare: y in F_q^x, flagged in the row):
//     sum_x chi(f_c(x)) = n_0 chi(c) + (Q - n_0) - 2 cnt_c - z_c,
//     #C_k(f_c) = Q + sum_x chi(f_c(x)) + 1 + chi(f(inf))          (Sec. 1.1).
// Members are counted exactly as Algorithm 1's evaluation loop counts them;
// only the work shared by the q members of a group is done once.
#pragma once
#include "count_common.cuh"

#include <algorithm>

namespace hwc {
namespace {

constexpr int kFanWarps = 8;          // warps per CTA of the fan-out kernels
constexpr uint32_t kChunkBlocks = 31; // 8-input blocks per lane before a flush (< 256 per plane set)

// CTAs per SM the register allocation aims at: 3 where the chain is short
// enough to stay in 80 registers without spilling, else 2
template <int D, int W>
constexpr int fan_min_ctas() { return (D <= 6 && W == 1) ? 3 : 2; }

__device__ __forceinline__ void csa(uint32_t &h, uint32_t &l, uint32_t a, uint32_t b, uint32_t c)
{
    const uint32_t u = a ^ b;
    h = (a & b) | (u & c);
    l = u ^ c;
}

// bit-sliced per-position counters of one 32-bit row word, counts < 256
struct Planes {
    uint32_t p[8];
};

// Horner in the log domain for h(x) = sum_{i>=LOW} c_i x^(i-LOW) with explicit
// zero handling; returns log h(x) or L when h(x) = 0.
template <int D>
struct LamV {
    uint32_t v[D + 1];
};

template <int D, int LOW, class Tab>
__device__ __noinline__ uint32_t slow_log_h(const Tab T, uint32_t L, uint32_t cap, const LamV<D> lamv,
                                            uint32_t nz, uint32_t j)
{
    const uint32_t(&lam)[D + 1] = lamv.v;
    uint32_t l = lam[D];
    bool zero = false;
#pragma unroll
    for (int i = D - 1; i >= LOW; --i) {
        if (!zero) l = addmod(l, j, L);
        if ((nz >> i) & 1u) {
            if (zero) {
                l = lam[i];
                zero = false;
            } else {
                const uint32_t n = addmod(l, L - lam[i], L);
                const uint32_t z = T[n];
                if (z >= cap) zero = true;
                else l = addmod(lam[i], z, L);
            }
        }
    }
    return zero ? L : l;
}

// Per-group, per-field constants of the h chain (uniform across the warp).
template <int D>
struct HChain {
    uint32_t base1;      // lam_D + (L - lam_{i1}): first index is base1 + g1*j (mod-free part)
    uint32_t g1;         // D - i1
    uint32_t dli[D];     // per position: lam_prev - lam_i (mod L)
    uint32_t gpi[D];     // per position: gap to the previous nonzero (0: no step)
    uint32_t lam_last;   // lam_{is}
    uint32_t tail;       // is: y = alpha^(lam_last + z + is*j)
    int dense;           // 2: positions 1..D-2 all nonzero and c_{D-1} = 0; 0: general
    bool none;           // h = c_D x^(D-1)
};

// LOW = 1: h over c_1..c_d (one-level fan-out); LOW = 2: v over c_2..c_d
template <int D, int LOW = 1>
__device__ __forceinline__ void make_hchain(HChain<D> &H, const uint32_t (&lam)[D + 1], uint32_t nz, uint32_t L)
{
    const uint32_t nzh = nz & ~((1u << LOW) - 1u);   // positions LOW..D-1
    H.none = nzh == 0;
    const int i1 = H.none ? 0 : 31 - __clz(nzh);
    const int is = H.none ? D : __ffs(nzh) - 1;
    H.g1 = (uint32_t)(D - i1);
    H.base1 = H.none ? 0 : lam[D] + (L - lam[i1]);
    H.lam_last = H.none ? lam[D] : lam[is];
    H.tail = (uint32_t)is;
    uint32_t lp = H.none ? 0 : lam[i1];
    int ip = i1;
#pragma unroll
    for (int i = D - 1; i >= 0; --i) {
        H.dli[i] = 0;
        H.gpi[i] = 0;
        if (i >= LOW && i < i1 && ((nzh >> i) & 1u)) {
            H.dli[i] = addmod(lp, L - lam[i], L);
            H.gpi[i] = (uint32_t)(ip - i);
            lp = lam[i];
            ip = i;
        }
    }
    const uint32_t full2 = ((1u << (D - 1)) - 1u) & ~((1u << LOW) - 1u);   // bits LOW..D-2
    H.dense = (nzh == full2) ? 2 : 0;
}

// chain steps for coefficient patterns with zeros below the lead (any gaps);
// out of line: such groups are a few percent of a family
template <int D, bool TRIPLE, int LOW, class Tab>
__device__ __noinline__ void general_chain(const Tab T, uint32_t L, uint32_t bar, uint32_t cap,
                                           const HChain<D> H, uint32_t xA, uint32_t xB, uint32_t &uA,
                                           uint32_t &uB)
{
#pragma unroll
    for (int i = D - 2; i >= LOW; --i) {
        if (H.gpi[i] == 0) continue;
        uint32_t sA, sB;
        if (H.gpi[i] == 1) {
            sA = xA;
            sB = xB;
        } else {
            sA = mulmod_small(H.gpi[i], xA, L, bar);
            sB = mulmod_small(H.gpi[i], xB, L, bar);
        }
        const uint32_t zA = T[uA], zB = T[uB];
        uA = chain_step<TRIPLE>(zA, H.dli[i], sA, L, cap);
        uB = chain_step<TRIPLE>(zB, H.dli[i], sB, L, cap);
    }
}

// log y for x = alpha^j (y = x^LOW h(x) = sum_{i>=LOW} c_i x^i), or L when
// y = 0; two x per lane.
template <int D, bool TRIPLE, class Tab, int LOW = 1>
__device__ __forceinline__ void log_y_pair(const Tab T, uint32_t L, uint32_t bar, const HChain<D> &H,
                                           const uint32_t (&lam)[D + 1], uint32_t nz, uint32_t xA,
                                           uint32_t xB, uint32_t &yA, uint32_t &yB)
{
    const uint32_t cap = TRIPLE ? 3 * L : 2 * L;
    if (H.none) {   // y = c_D x^D
        yA = addmod(lam[D], mulmod_small(D, xA, L, bar), L);
        yB = addmod(lam[D], mulmod_small(D, xB, L, bar), L);
        return;
    }
    uint32_t mA, mB;
    if (H.g1 == 2) {
        mA = min(2 * xA, 2 * xA - L);
        mB = min(2 * xB, 2 * xB - L);
    } else {
        mA = mulmod_small(H.g1, xA, L, bar);
        mB = mulmod_small(H.g1, xB, L, bar);
    }
    uint32_t uA = H.base1 + mA, uB = H.base1 + mB;   // < 3L
    if (!TRIPLE) {
        uA = min(uA, uA - L);
        uB = min(uB, uB - L);
    }
    if (H.dense == 2) {
#pragma unroll
        for (int i = D - 3; i >= LOW; --i) {
            const uint32_t zA = T[uA], zB = T[uB];
            uA = chain_step<TRIPLE>(zA, H.dli[i], xA, L, cap);
            uB = chain_step<TRIPLE>(zB, H.dli[i], xB, L, cap);
        }
    } else {
        general_chain<D, TRIPLE, LOW>(T, L, bar, cap, H, xA, xB, uA, uB);
    }
    const uint32_t zA = T[uA], zB = T[uB];
    // y = alpha^(lam_last + z + tail*j)
    uint32_t tA, tB;
    if (H.tail == 1) {
        tA = xA;
        tB = xB;
    } else {
        tA = mulmod_small(H.tail, xA, L, bar);
        tB = mulmod_small(H.tail, xB, L, bar);
    }
    yA = addmod(addmod(H.lam_last, zA, L), tA, L);
    yB = addmod(addmod(H.lam_last, zB, L), tB, L);
    const bool pA = zA >= cap, pB = zB >= cap;
    if (__any_sync(0xFFFFFFFFu, pA || pB)) {
        LamV<D> lv;
#pragma unroll
        for (int i = 0; i <= D; ++i) lv.v[i] = lam[i];
        if (pA) {
            const uint32_t lh = slow_log_h<D, LOW>(T, L, cap, lv, nz, xA);
            yA = lh == L ? L : addmod(lh, LOW == 1 ? xA : mulmod_small(LOW, xA, L, bar), L);
        }
        if (pB) {
            const uint32_t lh = slow_log_h<D, LOW>(T, L, cap, lv, nz, xB);
            yB = lh == L ? L : addmod(lh, LOW == 1 ? xB : mulmod_small(LOW, xB, L, bar), L);
        }
    }
}

// fan-out row of log y (W words); y = 0 gives an empty row and counts in n0;
// rows whose y lies in F_q^x add the zero position to zc (shared, per warp)
template <int W>
__device__ __forceinline__ void row_of(const uint8_t *rows, const uint8_t *zdig, uint32_t zdiv, uint32_t L,
                                       uint32_t y, bool valid, uint32_t (&m)[W], uint32_t &n0,
                                       uint32_t *zc)
{
    const bool zero_y = y >= L;
    const uint32_t yy = zero_y ? 0 : y;
    bool flag;
    if (W == 1) {
        const uint32_t r = reinterpret_cast<const uint32_t *>(rows)[yy];
        m[0] = r & 0x7FFFFFFFu;
        flag = r >> 31;
    } else {
        const uint2 r = reinterpret_cast<const uint2 *>(rows)[yy];
        m[0] = r.x;
        m[W - 1] = r.y & 0x7FFFFFFFu;
        flag = r.y >> 31;
    }
    const bool live = valid && !zero_y;
    if (!live) {
#pragma unroll
        for (int w = 0; w < W; ++w) m[w] = 0;
    }
    n0 += (valid && zero_y) ? 1u : 0u;
    // l / s for l a multiple of s = L/(q-1); zdiv = 0 encodes s = 1 (k = 1)
    if (live && flag) atomicAdd(&zc[zdig[zdiv ? __umulhi(yy, zdiv) : yy]], 1u);
}

// add 8 row words into the planes (carry-save tree, then ripple of the eights)
__device__ __forceinline__ void add8(Planes &P, const uint32_t (&a)[8])
{
    uint32_t tA, tB, fA, fB, e;
    csa(tA, P.p[0], P.p[0], a[0], a[1]);
    csa(tB, P.p[0], P.p[0], a[2], a[3]);
    csa(fA, P.p[1], P.p[1], tA, tB);
    csa(tA, P.p[0], P.p[0], a[4], a[5]);
    csa(tB, P.p[0], P.p[0], a[6], a[7]);
    csa(fB, P.p[1], P.p[1], tA, tB);
    csa(e, P.p[2], P.p[2], fA, fB);
#pragma unroll
    for (int b = 3; b < 8; ++b) {
        const uint32_t c = P.p[b] & e;
        P.p[b] ^= e;
        e = c;
    }
}

// sum the planes of the 32 lanes; lane c gets the count of bit position c.
// NB: planes 0..NB-1 are in use on entry (per-lane counts < 2^NB).
template <int NB>
__device__ __forceinline__ uint32_t reduce_planes(const uint32_t (&p)[8])
{
    uint32_t s[NB + 5];
#pragma unroll
    for (int b = 0; b < NB + 5; ++b) s[b] = b < NB ? p[b] : 0u;
#pragma unroll
    for (int lvl = 0; lvl < 5; ++lvl) {
        const int off = 16 >> lvl;
        uint32_t carry = 0;
#pragma unroll
        for (int b = 0; b <= NB + lvl; ++b) {
            const uint32_t o = __shfl_xor_sync(0xFFFFFFFFu, s[b], off);
            const uint32_t x = s[b] ^ o;
            const uint32_t nc = (s[b] & o) | (x & carry);
            s[b] = x ^ carry;
            carry = nc;
        }
    }
    const int lane = threadIdx.x & 31;
    uint32_t cnt = 0;
#pragma unroll
    for (int b = 0; b < NB + 5; ++b) cnt |= ((s[b] >> lane) & 1u) << b;
    return cnt;
}

template <int D>
__device__ __forceinline__ void decode_index(const KJob &J, uint64_t idx, uint32_t (&c)[D + 1])
{
    const uint32_t q = J.q;
    const bool all = J.kind == HWC_FAM_ALL_DEG;
    uint64_t r = idx;
#pragma unroll
    for (int i = 0; i < D; ++i) {
        if (i < D - 1 || all) {
            if (r >> 32) {
                c[i] = (uint32_t)(r % q);
                r /= q;
            } else {
                const uint32_t r32 = (uint32_t)r;
                c[i] = r32 % q;
                r = r32 / q;
            }
        }
    }
    if (all) {
        c[D] = 1 + (uint32_t)r;
    } else {
        c[D - 1] = 0;
        c[D] = 1;
    }
}

// square-freeness by Euclid's algorithm on gcd(f, f') with F_q digit tables
// (a*b, a-b, 1/a) in shared memory
template <int D>
__device__ bool squarefree_digits(const uint8_t *mulT, const uint8_t *subT, const uint8_t *invT,
                                  uint32_t q, uint32_t p, const uint32_t (&c)[D + 1])
{
    uint32_t P[2][D + 1];
    int dg[2];
#pragma unroll
    for (int i = 0; i <= D; ++i) P[0][i] = c[i];
    // f' = sum i c_i x^(i-1); the integer i is the digit (i mod p)
#pragma unroll
    for (int i = 1; i <= D; ++i) P[1][i - 1] = mulT[(i % p) * q + c[i]];
    P[1][D] = 0;
    dg[0] = D;
    dg[1] = D - 1;
    while (dg[0] >= 0 && P[0][dg[0]] == 0) --dg[0];
    while (dg[1] >= 0 && P[1][dg[1]] == 0) --dg[1];
    if (dg[1] < 0) return false;
    int a = 0, b = 1;
    while (dg[b] >= 0) {
        const int db = dg[b];
        const uint32_t il = invT[P[b][db]];
        for (int t = dg[a]; t >= db; --t) {
            const uint32_t at = P[a][t];
            if (!at) continue;
            const uint32_t cf = mulT[at * q + il];
            for (int i = 0; i <= db; ++i)
                P[a][t - db + i] = subT[P[a][t - db + i] * q + mulT[cf * q + P[b][i]]];
        }
        int da = db - 1;
        while (da >= 0 && P[a][da] == 0) --da;
        dg[a] = da;
        const int tmp = a;
        a = b;
        b = tmp;
    }
    return dg[a] == 0;
}

// per-member counts of one field for the whole group: lane c gets sum_x chi(f_c(x))
// for c = lane (and lane + 32), from n_0, the row-bit counts and z_c.  The
// points are x = alpha^j for j = pts[i], i < np (one per Frobenius orbit), or
// every j < L when pts is null.
template <int D, int W, bool TRIPLE, class Tab>
__device__ __forceinline__ void group_field(const Tab T, const KJob &J, int k, const uint8_t *smem,
                                            const HChain<D> &H, const uint32_t (&lam)[D + 1], uint32_t nz,
                                            uint32_t *zc, int lane, uint32_t &n0, uint32_t (&cnt)[W])
{
    const uint32_t L = J.L[k];
    const uint32_t *__restrict__ pts = J.reps[k];
    const uint32_t np = J.npts[k];
    auto point = [&](uint32_t i) -> uint32_t { return pts ? __ldg(pts + i) : i; };
    const uint8_t *rows = smem + J.row_off[k];
    const uint8_t *zdig = smem + J.zdig_off[k];
    const uint32_t zdiv = J.zdiv[k];
    const uint32_t bar = J.barrett[k];
    if (np <= 64) {   // few points (F_q, or a small orbit list): one pair of x per lane, counts < 4
        const uint32_t jA = lane, jB = lane + 32;
        const bool vA = jA < np, vB = jB < np;
        uint32_t yA, yB;
        log_y_pair<D, TRIPLE>(T, L, bar, H, lam, nz, vA ? point(jA) : 0, vB ? point(jB) : 0, yA, yB);
        uint32_t mA[W], mB[W];
        row_of<W>(rows, zdig, zdiv, L, yA, vA, mA, n0, zc);
        row_of<W>(rows, zdig, zdiv, L, yB, vB, mB, n0, zc);
#pragma unroll
        for (int w = 0; w < W; ++w) {
            uint32_t p2[8] = {mA[w] ^ mB[w], mA[w] & mB[w], 0, 0, 0, 0, 0, 0};
            cnt[w] += reduce_planes<2>(p2);
        }
        return;
    }
    for (uint32_t c0 = 0; c0 < np; c0 += kChunkBlocks * 256) {
        Planes P[W];
#pragma unroll
        for (int w = 0; w < W; ++w)
#pragma unroll
            for (int b = 0; b < 8; ++b) P[w].p[b] = 0;
        const uint32_t cend = min(np, c0 + kChunkBlocks * 256);
        for (uint32_t j0 = c0; j0 < cend; j0 += 256) {
            uint32_t a[W][8];
#pragma unroll
            for (int it = 0; it < 4; ++it) {
                const uint32_t jA = j0 + it * 64 + lane, jB = jA + 32;
                const bool vA = jA < cend, vB = jB < cend;
                uint32_t yA, yB;
                log_y_pair<D, TRIPLE>(T, L, bar, H, lam, nz, vA ? point(jA) : 0, vB ? point(jB) : 0, yA, yB);
                uint32_t mA[W], mB[W];
                row_of<W>(rows, zdig, zdiv, L, yA, vA, mA, n0, zc);
                row_of<W>(rows, zdig, zdiv, L, yB, vB, mB, n0, zc);
#pragma unroll
                for (int w = 0; w < W; ++w) {
                    a[w][2 * it] = mA[w];
                    a[w][2 * it + 1] = mB[w];
                }
            }
#pragma unroll
            for (int w = 0; w < W; ++w) add8(P[w], a[w]);
        }
        // per-lane counts are below 8 * blocks: fewer planes to add across lanes
        const uint32_t nblk = (cend - c0 + 255) / 256;
#pragma unroll
        for (int w = 0; w < W; ++w) {
            if (nblk <= 3) cnt[w] += reduce_planes<5>(P[w].p);
            else if (nblk <= 7) cnt[w] += reduce_planes<6>(P[w].p);
            else if (nblk <= 15) cnt[w] += reduce_planes<7>(P[w].p);
            else cnt[w] += reduce_planes<8>(P[w].p);
        }
    }
}

// one group of q members (c_0 = 0..q-1) for one warp
template <int D, int W>
__device__ __forceinline__ void process_group(const KJob &J, uint64_t gtile, const uint8_t *smem, uint32_t *zc, int lane,
                              WarpStats &st)
{
    constexpr int G = (D - 1) / 2;
    const uint32_t q = J.q;
    const uint64_t grp = J.first_group + gtile;
    const uint64_t base = grp * q;
    // coefficients c_1..c_D of the group (every lane decodes the same index)
    uint32_t c[D + 1];
    decode_index<D>(J, base, c);
    c[0] = 0;
    uint32_t nz = 0;
#pragma unroll
    for (int i = 1; i < D; ++i) nz |= (c[i] != 0 ? 1u : 0u) << i;

    const uint16_t *s16 = reinterpret_cast<const uint16_t *>(smem);
    const uint32_t *s32 = reinterpret_cast<const uint32_t *>(smem);
    const uint8_t *mulT = smem + J.fq_off;
    const uint8_t *subT = mulT + q * q;
    const uint8_t *invT = subT + q * q;

    // this lane's members: c_0 = lane (and lane + 32)
    bool valid[W], sqf[W];
    uint32_t anyv = 0, anys = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) {
        const uint32_t c0 = (uint32_t)lane + 32u * w;
        const uint64_t idx = base + c0;
        valid[w] = c0 < q && idx >= J.first && idx < J.first + J.count;
        sqf[w] = false;
        if (valid[w]) {
            uint32_t cm[D + 1];
#pragma unroll
            for (int i = 0; i <= D; ++i) cm[i] = c[i];
            cm[0] = c0;
            sqf[w] = squarefree_digits<D>(mulT, subT, invT, q, J.p, cm);
        }
        const unsigned vm = __ballot_sync(0xFFFFFFFFu, valid[w]);
        const unsigned sm = __ballot_sync(0xFFFFFFFFu, sqf[w]);
        anyv |= vm;
        anys |= sm;
        if (lane == 0) {
            st.examined += __popc(vm);
            st.sqf += __popc(sm);
        }
    }
    if ((J.unfiltered ? anyv : anys) == 0) {   // nothing to evaluate in this group
        if (J.member_counts) {
#pragma unroll
            for (int w = 0; w < W; ++w) {
                if (!valid[w]) continue;
                const uint64_t m = base + (uint32_t)lane + 32u * w - J.first;
#pragma unroll
                for (int k = 0; k < G; ++k) J.member_counts[m * G + k] = 0;
                J.member_sqf[m] = 0;
            }
        }
        return;
    }

    int E[W][G], Zr[W][G];   // per field: sum of chi and zeros over its points (x = 0 in field 1)
#pragma unroll
    for (int k = 0; k < G; ++k) {
        const uint32_t L = J.L[k];
        const uint32_t *coefk = s32 + J.coef_off[k];
        uint32_t lam[D + 1];
#pragma unroll
        for (int i = 0; i <= D; ++i) lam[i] = coefk[c[i]];
        HChain<D> H;
        make_hchain<D>(H, lam, nz, L);
        // clear the zero-correction counters of this warp
        zc[lane] = 0;
        zc[lane + 32] = 0;
        __syncwarp();
        uint32_t n0 = 0, cnt[W];
#pragma unroll
        for (int w = 0; w < W; ++w) cnt[w] = 0;
        const uint32_t kind = J.tab_kind[k];
        if (kind == kTabTripleSmem)
            group_field<D, W, true>(TabS{s16 + J.tab_off[k]}, J, k, smem, H, lam, nz, zc, lane, n0, cnt);
        else if (kind == kTabDoubleSmem)
            group_field<D, W, false>(TabS{s16 + J.tab_off[k]}, J, k, smem, H, lam, nz, zc, lane, n0, cnt);
        else
            group_field<D, W, false>(TabG{J.zech2w[k]}, J, k, smem, H, lam, nz, zc, lane, n0, cnt);
        // x = 0 (y = g(0) = 0) belongs to F_q, and to every field when every point is evaluated
        const uint32_t x0 = J.reps[k] == nullptr ? 1u : 0u;
        n0 = __reduce_add_sync(0xFFFFFFFFu, n0) + x0;
        const uint32_t npk = J.npts[k] + x0;   // points of the field, x = 0 included
        __syncwarp();
#pragma unroll
        for (int w = 0; w < W; ++w) {
            const uint32_t cc = (uint32_t)lane + 32u * w;
            const uint32_t lc = cc < q ? coefk[cc] : L;
            const int chi_c = (lc == L) ? 0 : ((lc & 1u) ? -1 : 1);
            // y = 0: f_c = c; y = -c != 0: f_c = 0; else chi(y + c) from the row bits
            E[w][k] = (int)n0 * chi_c + (int)(npk - n0) - 2 * (int)cnt[w] - (int)zc[cc];
            Zr[w][k] = cc == 0 ? (int)n0 : (int)zc[cc];
        }
        __syncwarp();   // zc is cleared for the next field
    }
    // #C_k = Q_k + S_k + 1 + chi(c_{2g+2})
    int32_t N[W][G];
#pragma unroll
    for (int w = 0; w < W; ++w) {
        int Sk[G];
        orbit_combine<G>(J, E[w], Zr[w], Sk);
#pragma unroll
        for (int k = 0; k < G; ++k) {
            int inf = 1;
            if (D == 2 * G + 2) inf += (s32[J.coef_off[k] + c[D]] & 1u) ? -1 : 1;
            N[w][k] = (int32_t)J.Q[k] + Sk[k] + inf;
        }
    }

#pragma unroll
    for (int w = 0; w < W; ++w) {
        const uint32_t c0 = (uint32_t)lane + 32u * w;
        if (J.member_counts) {
            if (valid[w]) {
                const uint64_t m = base + c0 - J.first;
#pragma unroll
                for (int k = 0; k < G; ++k) J.member_counts[m * G + k] = (sqf[w] || J.unfiltered) ? N[w][k] : 0;
                J.member_sqf[m] = sqf[w] ? 1 : 0;
            }
            continue;
        }
        unsigned long long key = 0;
#pragma unroll
        for (int k = 0; k < G; ++k) {
            const int a = (int)J.Q[k] + 1 - N[w][k];   // eq. 1.1
            key |= (unsigned long long)((uint32_t)(a + 32768) & 0xFFFFu) << (16 * k);
        }
        const unsigned smask = __ballot_sync(0xFFFFFFFFu, sqf[w]);
        if (sqf[w]) {
            const unsigned peers = __match_any_sync(smask, key);
            if (lane == __ffs(peers) - 1) hist_insert(J, key, __popc(peers));
        }
    }
}

template <int D, int W>
__global__ void __launch_bounds__(kFanWarps * 32, fan_min_ctas<D, W>()) k_fan_persistent(const KJob *__restrict__ jobs,
                                                                   const uint64_t *__restrict__ item_start,
                                                                   uint32_t n_jobs, uint64_t n_items,
                                                                   unsigned long long *counter,
                                                                   uint32_t item_tiles)
{
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ uint32_t zc_all[kFanWarps][64];
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
        const uint64_t t0 = (item - item_start[jb]) * item_tiles;
        const uint64_t t1 = min(t0 + item_tiles, J.n_tiles);
        for (uint64_t t = t0 + warp; t < t1; t += nw) process_group<D, W>(J, t, smem, zc_all[warp], lane, st);
        __syncthreads();
    }
    if (cur >= 0) flush_stats(jobs[cur], st, lane);
}

template <int D, int W>
const void *fan_pick(bool persistent)
{
    return persistent ? (const void *)k_fan_persistent<D, W> : nullptr;
}

}  // namespace
}  // namespace hwc
