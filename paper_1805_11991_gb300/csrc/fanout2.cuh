// fanout2.cuh -- two-level (c_1, c_0) fan-out count kernel for enumerated
// families with q <= 31; instantiated per degree in fan2_a.cu and fan2_b.cu.
//
// q^2 consecutive members of a family differ only in c_1 = b and c_0 = c:
// f_{b,c}(x) = u(x) + b x + c with u(x) = sum_{i>=2} c_i x^i.  One warp takes
// such a group.  For 64 points x = alpha^j at a time the warp evaluates u(x)
// by the Zech-index Horner chain over c_2..c_d (one chain per x, shared by all
// q^2 members) and stages log u(x) in shared memory.  Each lane owns one value
// of b (several lanes per b when q < 16, splitting the points) and, per point,
// does one Zech addition, y_b = u + b x = b x (1 + u / (b x)) (eq. 2.1), and
// reads the fan-out row of y_b: its q bits say chi(y_b + c) = -1 for every
// c at once.  A lane sums its rows per bit position with bit-sliced
// carry-save counters and from time to time adds the per-position counts
// into the group's (b, c) accumulators in shared memory.  With n_0(b) the
// number of x with y_b(x) = 0 (x = 0 included) and z(b, c) the rare x with
// y_b(x) = -c != 0:
//     sum_x chi(f_{b,c}(x)) = n_0 chi(c) + (Q - n_0) - 2 cnt(b, c) - z(b, c),
//     #C_k(f_{b,c}) = Q + sum_x chi(f_{b,c}(x)) + 1 + chi(f(inf))   (Sec. 1.1).
// Per point and member this is 1/q Zech additions and one row bit; the chain
// for u and every per-group cost are shared by q^2 members.  z(b, c) is
// counted directly per point for g <= 2 (fan2_zero_digits: one b per point
// outside F_q) and through the lanes' queues of flagged rows for g >= 3.
#pragma once
#include "fanout.cuh"

namespace hwc {
namespace {

constexpr int kFan2Warps = 4;                 // smallest block (warps)
constexpr int kFan2Planes = 10;               // per-lane counts < 1024 between flushes
// 8-input blocks per lane between flushes: a flush follows as soon as the
// count reaches 124, and at most 4 blocks are added between the tests, so
// no position exceeds 127 x 8 = 1016 < 1024
constexpr uint32_t kFan2FlushBlocks = 124;

// add 8 row words into the carry-save planes 0..2 (ones, twos, fours); returns
// the carry of weight 8, to be added into plane 3 and up by the caller
__device__ __forceinline__ uint32_t csa8(uint32_t (&P)[kFan2Planes], const uint32_t (&a)[8])
{
    uint32_t tA, tB, fA, fB, e;
    csa(tA, P[0], P[0], a[0], a[1]);
    csa(tB, P[0], P[0], a[2], a[3]);
    csa(fA, P[1], P[1], tA, tB);
    csa(tA, P[0], P[0], a[4], a[5]);
    csa(tB, P[0], P[0], a[6], a[7]);
    csa(fB, P[1], P[1], tA, tB);
    csa(e, P[2], P[2], fA, fB);
    return e;
}

// add a carry word of weight 2^B0 into planes B0.. (ripple)
template <int B0>
__device__ __forceinline__ void ripple(uint32_t (&P)[kFan2Planes], uint32_t e)
{
#pragma unroll
    for (int b = B0; b < kFan2Planes; ++b) {
        const uint32_t c = P[b] & e;
        P[b] ^= e;
        e = c;
    }
}

// add 8 row words into 10 bit-sliced planes (carry-save tree, ripple of the eights)
__device__ __forceinline__ void add8_p10(uint32_t (&P)[kFan2Planes], const uint32_t (&a)[8])
{
    ripple<3>(P, csa8(P, a));
}

// add the per-position counts of the planes into the lane's row (2 per row
// bit), clear the planes
__device__ __forceinline__ void flush_planes(uint32_t (&P)[kFan2Planes], uint16_t *acc_row, uint32_t q, bool role)
{
    if (role) {
        for (uint32_t c = 0; c < q; ++c) {
            uint32_t v = 0;
#pragma unroll
            for (int b = 0; b < kFan2Planes; ++b) v |= ((P[b] >> c) & 1u) << b;
            if (v) acc_row[c] = (uint16_t)(acc_row[c] + 2 * v);
        }
    }
#pragma unroll
    for (int b = 0; b < kFan2Planes; ++b) P[b] = 0;
}

// the lane's queued points with y in F_q (y + c = 0 for one digit c): z(b, c) += 1.
// Entries are staged row indices: i < L + 8 stands for log y = i mod L,
// L + 8 for y = 0 (digit 0).  The lane's entries sit at lane, lane + 32, ...;
// qn = lane + 32 * (number of entries).
__device__ __forceinline__ void drain_queue(const uint16_t *rq, uint32_t qn, int lane, const uint8_t *zdig,
                                            uint32_t zdiv, uint32_t L, uint16_t *acc_row, uint32_t zw)
{
    // selects, no branches in the body
    const uint32_t zrow = L + kFan2ZeroRow;
    for (uint32_t i = (uint32_t)lane; i < qn; i += 32) {
        uint32_t l = rq[i];
        const bool zr = l == zrow;
        if (L >= kFan2ZeroRow) l = min(l, l - L);   // rows [L, L + 8) stand for l - L
        else l %= L;                               // fields of fewer than 8 nonzero elements
        // in bounds for zr too: index <= 8 < 16 <= zdig bytes
        const uint32_t d = zdig[zdiv ? __umulhi(l, zdiv) : l];
        const uint32_t di = zr ? 0u : d;
        acc_row[di] = (uint16_t)(acc_row[di] + zw);
    }
}

// z(b, c) += 1 in the group's accumulator rows (row b of chunk 0, column c):
// one shared atomic on the u32 word that holds the u16 entry; zw = 1, or
// 1 + 2^s where the field's zeros are also kept apart in bits s..
__device__ __forceinline__ void zinc(uint32_t *acc32, uint32_t q, uint32_t b, uint32_t c, uint32_t zw)
{
    const uint32_t i = b * q + c;
    atomicAdd(acc32 + (i >> 1), zw << ((i & 1u) << 4));
}

// Zero digits of one batch of points counted directly, for F_q (k = 1) and
// F_{q^2} (k = 2), instead of flagging rows lane by lane: z(b, c) += 1 for every
// x of the batch and every b with y_b(x) = u(x) + b x in F_q, c = -y_b(x).
//   x in F_q: u(x) is in F_q too (the c_i are), so every b counts, with
//     c = -(u + b x);
//   x in F_{q^2} \ F_q: with u = u0 + u1 alpha, x = x0 + x1 alpha (x1 != 0),
//     u + b x lies in F_q for exactly one b, b = -u1 / x1 = (-u1) A, and then
//     c = -(u0 + b x0) = (-u0) + (-u1) B with A = 1/x1, B = -x0/x1.
// KF = 1: all points are in F_q, whose digits come from zdig (zdig[l] = -alpha^l).
// KF = 2: coordinate table crd[l] = -y0 | -y1 << 8 | A << 16 | B << 24 (A = 0,
// B = -y0 for elements of F_q, the points alpha^j with j = 0 mod (q + 1));
// jq walks those multiples of q + 1 across batches (consecutive points only:
// with one point per Frobenius orbit of degree 2 no point lies in F_q).
// Us holds log u(x) (>= L for u = 0) of the batch's nb points from j0; the
// lane's own two points are xA, xB (validity vA, vB) with u = uA, uB.
template <int KF, bool REPS>
__device__ __forceinline__ void fan2_zero_digits(const uint32_t *Us, uint32_t j0, uint32_t nb, uint32_t L,
                                                 uint32_t q, int lane, uint32_t xA, uint32_t xB, bool vA, bool vB,
                                                 uint32_t uA, uint32_t uB, const uint8_t *fq, const uint8_t *zdig,
                                                 const uint32_t *crd, uint32_t *acc32, uint32_t &jq, uint32_t zw)
{
    const uint32_t qq = q * q;
    const uint8_t *mulT = fq, *addT = fq + 2 * qq + q;
    if constexpr (KF == 1) {
        // -(u + b x) = (-u) + b (-x)
        for (uint32_t i = 0; i < nb; ++i) {
            const uint32_t lu = Us[i];
            const uint32_t nu = lu < L ? zdig[lu] : 0u, nx = zdig[j0 + i];
            if ((uint32_t)lane < q)
                zinc(acc32, q, (uint32_t)lane, addT[nu * q + mulT[(uint32_t)lane * q + nx]], zw);
        }
    } else {
    // both loads first
    const uint32_t tA = crd[vA ? xA : 0u], tB = crd[vB ? xB : 0u];
    uint32_t cA = crd[uA < L ? uA : 0u], cB = crd[uB < L ? uB : 0u];
    cA = uA < L ? cA : 0u;
    cB = uB < L ? cB : 0u;
    if (vA && (tA & 0xFF0000u))
        zinc(acc32, q, mulT[((cA >> 8) & 0xFFu) * q + ((tA >> 16) & 0xFFu)],
             addT[(cA & 0xFFu) * q + mulT[((cA >> 8) & 0xFFu) * q + (tA >> 24)]], zw);
    if (vB && (tB & 0xFF0000u))
        zinc(acc32, q, mulT[((cB >> 8) & 0xFFu) * q + ((tB >> 16) & 0xFFu)],
             addT[(cB & 0xFFu) * q + mulT[((cB >> 8) & 0xFFu) * q + (tB >> 24)]], zw);
    if (!REPS) {
        for (; jq < j0 + nb; jq += q + 1) {   // x in F_q: u = u0, c = -u0 + b (-x0)
            const uint32_t lu = Us[jq - j0];
            const uint32_t n0 = lu < L ? (crd[lu] & 0xFFu) : 0u, nx = crd[jq] >> 24;
            if ((uint32_t)lane < q)
                zinc(acc32, q, (uint32_t)lane, addT[n0 * q + mulT[(uint32_t)lane * q + nx]], zw);
        }
    }
    }
}

// queue the block's flagged points (row top bit: y in F_q, rare for k >= 3):
// one test of the OR of the 8 rows, the per-point stores only when set
__device__ __forceinline__ void queue_flagged(const uint32_t (&a)[8], const uint32_t (&ly)[8], uint16_t *rq,
                                              uint32_t &qn)
{
    const uint32_t any = (a[0] | a[1] | a[2] | a[3]) | (a[4] | a[5] | a[6] | a[7]);
    if ((int)any < 0) {
#pragma unroll
        for (int v = 0; v < 8; ++v)
            if ((int)a[v] < 0) {
                rq[qn] = (uint16_t)ly[v];
                qn += 32;
            }
    }
}

// One block of 8 consecutive points x = alpha^(j0 + i) for lane (b, s), with
// lb = log(b x) of the first point reduced mod L (later points lb + v, not
// reduced).  Phases over the 8 points so that their lookups overlap: staged
// log u -> Zech addition y_b = u + b x = b x (1 + u / (b x)) (eq. 2.1) ->
// fan-out row of y_b.  Row bit c is [chi(y_b + c) = -1]; the top bit flags
// y_b in F_q (y_b = 0 included), whose zero digit goes to the lane's queue.
// The row's top bit is counted too, in a position no member reads.
// GEN: points outside okm are dropped, and u may be 0.  QUEUE: queue the
// flagged points (fields whose zero digits are not counted directly).
template <bool GEN, bool QUEUE, class Tab, class RowT>
__device__ __forceinline__ void fan2_block(const Tab T, const RowT *__restrict__ rows, const uint32_t *Us,
                                           uint32_t L, uint32_t lb, bool b0, uint32_t okm, uint16_t *rq,
                                           uint32_t &qn, uint32_t (&a)[8])
{
    const uint4 w0 = *reinterpret_cast<const uint4 *>(Us);
    const uint4 w1 = *reinterpret_cast<const uint4 *>(Us + 4);
    const uint32_t U[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
    // staged Zech index of log u - log(b x) + L: in [58, 2L + 64]
    const uint32_t C = L + kFan2Prefix - lb;
    uint32_t ly[8];
#pragma unroll
    for (int v = 0; v < 8; ++v) {
        const uint32_t z = T.at(U[v] + C - v);
        uint32_t t = lb + v + z;          // < 2L + 6, or >= 65535 when u + b x = 0
        t = min(t, t - L);                // congruent mod L, < L + 6; poisoned: >= L + 8
        t = min(t, L + kFan2ZeroRow);     // row L + 8: y = 0
        if (GEN) t = (U[v] >= L) ? lb + v : t;   // u = 0: y = b x
        if (GEN) ly[v] = b0 ? (U[v] >= L ? L + kFan2ZeroRow : U[v]) : t;
        else ly[v] = b0 ? U[v] : t;       // b = 0: y = u
    }
    // all 8 row loads before any queue store (a store may alias later loads)
#pragma unroll
    for (int v = 0; v < 8; ++v) a[v] = (uint32_t)(int32_t)rows[ly[v]];   // int16 rows: the flag fills bits 15..31
#pragma unroll
    for (int v = 0; v < 8; ++v)
        if (GEN && !((okm >> v) & 1u)) a[v] = 0u;
    if (QUEUE) queue_flagged(a, ly, rq, qn);
}

// One block of 8 orbit points for lane (b, s): the staged log u(x) (U) and
// d = log u - log x (D) of each point.  y_b = u + b x = u (1 + b x / u), so
// log y_b = log u + Z(log b - d) (eq. 2.1): one Zech read at lam_b - d and one
// fan-out row per point, as in fan2_block, with the per-point log x folded
// into d.  u = 0 (GEN only) is staged as U >= L and D = -log x, where
// y_b = b x.
template <bool GEN, bool QUEUE, class Tab, class RowT>
__device__ __forceinline__ void fan2_block_reps(const Tab T, const RowT *__restrict__ rows, const uint32_t *Us,
                                                const uint32_t *Ds, uint32_t L, uint32_t lam_b, bool b0,
                                                uint32_t okm, uint16_t *rq, uint32_t &qn, uint32_t (&a)[8])
{
    const uint4 w0 = *reinterpret_cast<const uint4 *>(Us);
    const uint4 w1 = *reinterpret_cast<const uint4 *>(Us + 4);
    const uint4 d0 = *reinterpret_cast<const uint4 *>(Ds);
    const uint4 d1 = *reinterpret_cast<const uint4 *>(Ds + 4);
    const uint32_t U[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
    const uint32_t Dv[8] = {d0.x, d0.y, d0.z, d0.w, d1.x, d1.y, d1.z, d1.w};
    // staged Zech index of lam_b - d + L: in [1 + 64, 2L + 64)
    const uint32_t C = lam_b + L + kFan2Prefix;
    uint32_t ly[8];
#pragma unroll
    for (int v = 0; v < 8; ++v) {
        const uint32_t z = T.at(C - Dv[v]);
        uint32_t t = U[v] + z;            // < 2L, or >= 65535 when u + b x = 0
        t = min(t, t - L);                // < L; poisoned: >= L + 8
        t = min(t, L + kFan2ZeroRow);     // row L + 8: y = 0
        if (GEN) {
            uint32_t bx = lam_b + L - Dv[v];   // u = 0: y = b x, log in (0, 2L)
            bx = min(bx, bx - L);
            t = (U[v] >= L) ? bx : t;
            ly[v] = b0 ? (U[v] >= L ? L + kFan2ZeroRow : U[v]) : t;
        } else {
            ly[v] = b0 ? U[v] : t;        // b = 0: y = u
        }
    }
#pragma unroll
    for (int v = 0; v < 8; ++v) a[v] = (uint32_t)(int32_t)rows[ly[v]];   // int16 rows: the flag fills bits 15..31
#pragma unroll
    for (int v = 0; v < 8; ++v)
        if (GEN && !((okm >> v) & 1u)) a[v] = 0u;
    if (QUEUE) queue_flagged(a, ly, rq, qn);
}

// points of one field for the whole group (all q^2 members), lane role (b, s)
// The chain constants (lam_i and the h chain) come from the warp's shared
// parameters at every batch: the main loop keeps no registers for them.
// KF = 0: zero digits through the lanes' queues; KF = 1, 2: counted directly
// per batch (fan2_zero_digits).  REPS: the points are the field's orbit list
// J.reps[k] (J.npts[k] of them), else every x = alpha^j, j < L.  A zero of
// f_{b,c} adds zw to its accumulator (1, or 1 + 2^s to keep the field's zeros
// apart in bits s..).
template <int D, bool TRIPLE, bool PAD, int KF, bool REPS, class RowT = uint32_t>
__device__ __forceinline__ void group2_field(const KJob &J, int k, const uint8_t *smem, const HChain<D> *gH,
                                             const uint32_t *glam, uint32_t nz, uint32_t *Us, uint32_t *Ds,
                                             uint16_t *acc, uint16_t *acc_row, uint16_t *rq, int lane, bool role,
                                             uint32_t b, uint32_t s, uint32_t S, uint32_t zw)
{
    constexpr bool QUEUE = KF == 0;
    const TabP<PAD> T{reinterpret_cast<const uint16_t *>(smem) + J.tab_off[k]};
    const uint32_t L = J.L[k];
    const uint32_t bar = J.barrett[k];
    const RowT *rows = reinterpret_cast<const RowT *>(smem + J.row_off[k]);   // [L + 9]
    const uint8_t *zdig = smem + J.zdig_off[k];
    const uint32_t zdiv = J.zdiv[k];
    const uint32_t *coefk = reinterpret_cast<const uint32_t *>(smem) + J.coef_off[k];
    const uint32_t lam_b = (b != 0) ? coefk[b] : 0u;   // log b
    const bool b0 = b == 0;
    const bool pow2S = S == 1 || S == 2 || S == 4 || S == 8;   // 64 / S points per lane, a multiple of 8
    const uint32_t *__restrict__ pts = J.reps[k];
    const uint32_t np = REPS ? J.npts[k] : L;
    uint32_t P[kFan2Planes];
#pragma unroll
    for (int p = 0; p < kFan2Planes; ++p) P[p] = 0;
    uint32_t nblk = 0, qn = (uint32_t)lane, jq = 0;
    const uint32_t *crd = reinterpret_cast<const uint32_t *>(smem + J.coord_off);
    // orbit points of the next batch, loaded one batch ahead (global memory)
    uint32_t nxA = 0, nxB = 0;
    if (REPS) {
        nxA = __ldg(pts + min((uint32_t)lane, np - 1));
        nxB = __ldg(pts + min(32u + lane, np - 1));
    }
    for (uint32_t j0 = 0; j0 < np; j0 += 64) {
        // log u(x) for the batch, two points per lane, staged for all lanes
        const uint32_t iA = j0 + lane, iB = j0 + 32 + lane;
        const bool vA = iA < np, vB = iB < np;
        uint32_t xA = vA ? iA : 0, xB = vB ? iB : 0;
        if (REPS) {
            xA = nxA;   // loaded from a clamped index: a valid point for invalid lanes too
            xB = nxB;
            if (j0 + 64 < np) {
                nxA = __ldg(pts + min(j0 + 64 + lane, np - 1));
                nxB = __ldg(pts + min(j0 + 96 + lane, np - 1));
            }
        }
        uint32_t uA, uB;
        {
            const HChain<D> H = *gH;
            uint32_t lam[D + 1];
#pragma unroll
            for (int i = 0; i <= D; ++i) lam[i] = glam[i];
            log_y_pair<D, TRIPLE, TabP<PAD>, 2>(T, L, bar, H, lam, nz, xA, xB, uA, uB);
        }
        Us[lane] = uA;
        Us[32 + lane] = uB;
        if (REPS) {   // d = log u - log x (mod L); u = 0: d = -log x
            Ds[lane] = uA < L ? (uA >= xA ? uA - xA : uA + L - xA) : (xA ? L - xA : 0u);
            Ds[32 + lane] = uB < L ? (uB >= xB ? uB - xB : uB + L - xB) : (xB ? L - xB : 0u);
        }
        const bool uzero = __any_sync(0xFFFFFFFFu, uA >= L || uB >= L);
        __syncwarp();
        const uint32_t nb = min(64u, np - j0);   // points in this batch
        if (!QUEUE) {   // atomics here, plain row updates (flushes) after the barrier
            fan2_zero_digits<KF == 0 ? 1 : KF, REPS>(Us, j0, nb, L, J.q, lane, xA, xB, vA, vB, uA, uB,
                                                     smem + J.fq_off, zdig, crd, reinterpret_cast<uint32_t *>(acc),
                                                     jq, zw);
            __syncwarp();
        }
        if (pow2S && S <= 2 && nb == 64 && !uzero) {
            // 32 or 64 points per lane: steps of 4 blocks, whose eights meet in
            // carry-save planes 3 and 4 before one ripple of weight 32
            const uint32_t per = 64 / S, i0 = s * per;
            uint32_t lb = REPS ? 0u : addmod(lam_b, j0 + i0, L);
            auto blk = [&](uint32_t t0) -> uint32_t {
                uint32_t a[8];
                if (REPS) fan2_block_reps<false, QUEUE>(T, rows, Us + i0 + t0, Ds + i0 + t0, L, lam_b, b0, 0u, rq, qn, a);
                else fan2_block<false, QUEUE>(T, rows, Us + i0 + t0, L, lb, b0, 0u, rq, qn, a);
                if (!REPS) lb = addmod(lb, 8u % L, L);
                const uint32_t e = csa8(P, a);
                if (QUEUE && __any_sync(0xFFFFFFFFu, qn >= 32 * (kFan2Queue - 8 + 1))) {   // room for fewer than 8 more
                    drain_queue(rq, qn, lane, zdig, zdiv, L, acc_row, zw);
                    qn = (uint32_t)lane;
                }
                return e;
            };
            for (uint32_t t0 = 0; t0 < per; t0 += 32) {
                uint32_t s16a, s16b, s32;
                const uint32_t e0 = blk(t0);
                const uint32_t e1 = blk(t0 + 8);
                csa(s16a, P[3], P[3], e0, e1);
                const uint32_t e2 = blk(t0 + 16);
                const uint32_t e3 = blk(t0 + 24);
                csa(s16b, P[3], P[3], e2, e3);
                csa(s32, P[4], P[4], s16a, s16b);
                ripple<5>(P, s32);
                nblk += 4;
                if (nblk >= kFan2FlushBlocks) {
                    flush_planes(P, acc_row, J.q, true);
                    nblk = 0;
                }
            }
        } else if (pow2S && nb == 64 && !uzero) {
            const uint32_t per = 64 / S, i0 = s * per;
            uint32_t lb = REPS ? 0u : addmod(lam_b, j0 + i0, L);
            for (uint32_t t0 = 0; t0 < per; t0 += 8) {
                uint32_t a[8];
                if (REPS) fan2_block_reps<false, QUEUE>(T, rows, Us + i0 + t0, Ds + i0 + t0, L, lam_b, b0, 0u, rq, qn, a);
                else fan2_block<false, QUEUE>(T, rows, Us + i0 + t0, L, lb, b0, 0u, rq, qn, a);
                if (!REPS) lb = addmod(lb, 8u % L, L);
                add8_p10(P, a);
                if (++nblk >= kFan2FlushBlocks) {
                    flush_planes(P, acc_row, J.q, true);
                    nblk = 0;
                }
                if (QUEUE && __any_sync(0xFFFFFFFFu, qn >= 32 * (kFan2Queue - 8 + 1))) {   // room for fewer than 8 more
                    drain_queue(rq, qn, lane, zdig, zdiv, L, acc_row, zw);
                    qn = (uint32_t)lane;
                }
            }
        } else {
            // lane chunks of a multiple of 8 points; reads past 64 hit the
            // zeroed slack of U and D and are masked
            const uint32_t per = (((nb + S - 1) / S) + 7) & ~7u, i0 = s * per;
            uint32_t lb = REPS ? 0u : addmod(lam_b, (j0 + i0) % L, L);
            for (uint32_t t0 = 0; t0 < per; t0 += 8) {
                const int nv = role ? min(8, max(0, (int)nb - (int)(i0 + t0))) : 0;
                const uint32_t okm = (1u << nv) - 1u;
                uint32_t a[8];
                if (REPS) fan2_block_reps<true, QUEUE>(T, rows, Us + i0 + t0, Ds + i0 + t0, L, lam_b, b0, okm, rq, qn, a);
                else fan2_block<true, QUEUE>(T, rows, Us + i0 + t0, L, lb, b0, okm, rq, qn, a);
                if (!REPS) lb = addmod(lb, 8u % L, L);
                add8_p10(P, a);
                if (++nblk >= kFan2FlushBlocks) {
                    flush_planes(P, acc_row, J.q, true);
                    nblk = 0;
                }
                if (QUEUE && __any_sync(0xFFFFFFFFu, qn >= 32 * (kFan2Queue - 8 + 1))) {   // room for fewer than 8 more
                    drain_queue(rq, qn, lane, zdig, zdiv, L, acc_row, zw);
                    qn = (uint32_t)lane;
                }
            }
        }
        __syncwarp();   // U is rewritten by the next batch
    }
    flush_planes(P, acc_row, J.q, true);
    if (QUEUE) drain_queue(rq, qn, lane, zdig, zdiv, L, acc_row, zw);
}

// group2_field for the field's Zech layout (tripled or doubled, padded or not)
// and point set (orbit list or every point)
template <int D, int KF>
__device__ __forceinline__ void group2_field_tabs(const KJob &J, int k, bool tri, const uint8_t *smem,
                                                  const HChain<D> *gH, const uint32_t *glam, uint32_t nz,
                                                  uint32_t *Us, uint32_t *Ds, uint16_t *acc, uint16_t *acc_row,
                                                  uint16_t *rq, int lane, bool role, uint32_t b, uint32_t s,
                                                  uint32_t S, uint32_t zw)
{
#define HWC_G2F(TRI, PAD, REPS)                                                                             \
    group2_field<D, TRI, PAD, KF, REPS>(J, k, smem, gH, glam, nz, Us, Ds, acc, acc_row, rq, lane, role, b, s, S, \
                                        zw)
    if constexpr (D >= 9 && KF == 0) {   // g = 4: int16 rows (doubled Zech layout, orbit points)
        if (J.row16[k]) {
            if (J.tab_pad[k])
                group2_field<D, false, true, 0, true, int16_t>(J, k, smem, gH, glam, nz, Us, Ds, acc, acc_row, rq,
                                                               lane, role, b, s, S, zw);
            else
                group2_field<D, false, false, 0, true, int16_t>(J, k, smem, gH, glam, nz, Us, Ds, acc, acc_row, rq,
                                                                lane, role, b, s, S, zw);
            return;
        }
    }
    if (KF != 1 && J.reps[k]) {   // field 1 (KF = 1) takes every point
        if (J.tab_pad[k]) {
            if (tri) HWC_G2F(true, true, true);
            else HWC_G2F(false, true, true);
        } else {
            if (tri) HWC_G2F(true, false, true);
            else HWC_G2F(false, false, true);
        }
    } else {
        if (J.tab_pad[k]) {
            if (tri) HWC_G2F(true, true, false);
            else HWC_G2F(false, true, false);
        } else {
            if (tri) HWC_G2F(true, false, false);
            else HWC_G2F(false, false, false);
        }
    }
#undef HWC_G2F
}

// Square-freeness of the q members f_c = g_b + c (c in F_q) that share
// g_b(x) = u(x) + b x.  They share f' = w = u' + b, and gcd(f_c, w) != 1 exactly
// when some root theta of w has g_b(theta) = -c.  The characteristic polynomial
// of multiplication by g_b on F_q[x]/(w) is prod_theta (t - g_b(theta)) over the
// roots of w with multiplicity, so f_c is square-free iff chi(-c) != 0 (for
// deg w >= 1; w = 0 means f' = 0, never square-free; w a nonzero constant
// means always square-free).  chi comes from a Hessenberg form (similarity
// transforms) and the Hessenberg recurrence.  F_q arithmetic on digits with
// the mul / sub / inv tables.  Returns the mask of square-free c (bit c).
template <int D>
__device__ __noinline__ uint32_t sqf_mask_for_b(const uint8_t *mulT, const uint8_t *subT, const uint8_t *invT,
                                                const uint8_t *addT, uint32_t q, uint32_t p, const uint32_t *cg,
                                                uint32_t b)
{
    // digits fit a byte (q <= 31): byte arrays keep the lane's local
    // footprint small
    constexpr int MX = D - 1;   // deg w <= D - 1
    auto mul = [&](uint32_t x, uint32_t y) -> uint32_t { return mulT[x * q + y]; };
    auto sub = [&](uint32_t x, uint32_t y) -> uint32_t { return subT[x * q + y]; };
    auto add = [&](uint32_t x, uint32_t y) -> uint32_t { return addT[x * q + y]; };
    const uint32_t all = (q >= 32) ? 0xFFFFFFFFu : ((1u << q) - 1u);
    // w = f' = b + sum_{i>=2} (i mod p) c_i x^(i-1)
    uint8_t w[MX + 1];
    w[0] = (uint8_t)b;
    for (int i = 2; i <= D; ++i) w[i - 1] = (uint8_t)mul(i % p, cg[i]);
    int m = MX;
    while (m >= 0 && w[m] == 0) --m;
    if (m < 0) return 0u;
    if (m == 0) return all;
    const uint32_t wi = invT[w[m]];
    for (int i = 0; i <= m; ++i) w[i] = (uint8_t)mul(w[i], wi);   // monic
    // r = g_b mod w, g_b = b x + sum_{i>=2} c_i x^i
    uint8_t r[D + 1];
    r[0] = 0;
    r[1] = (uint8_t)b;
    for (int i = 2; i <= D; ++i) r[i] = (uint8_t)cg[i];
    for (int t = D; t >= m; --t) {
        const uint32_t cf = r[t];
        if (!cf) continue;
        r[t] = 0;
        for (int i = 0; i < m; ++i) r[t - m + i] = (uint8_t)sub(r[t - m + i], mul(cf, w[i]));
    }
    // H[i][j]: coefficient i of g_b x^j mod w
    uint8_t H[MX][MX];
    for (int j = 0; j < m; ++j) {
        for (int i = 0; i < m; ++i) H[i][j] = r[i];
        const uint32_t top = r[m - 1];
        for (int i = m - 1; i >= 1; --i) r[i] = (uint8_t)sub(r[i - 1], mul(top, w[i]));
        r[0] = (uint8_t)sub(0, mul(top, w[0]));
    }
    // upper Hessenberg form by similarity
    for (int j = 0; j + 2 < m; ++j) {
        int piv = -1;
        for (int i = j + 1; i < m; ++i)
            if (H[i][j]) { piv = i; break; }
        if (piv < 0) continue;
        if (piv != j + 1) {
            for (int k = 0; k < m; ++k) { const uint8_t t = H[piv][k]; H[piv][k] = H[j + 1][k]; H[j + 1][k] = t; }
            for (int k = 0; k < m; ++k) { const uint8_t t = H[k][piv]; H[k][piv] = H[k][j + 1]; H[k][j + 1] = t; }
        }
        const uint32_t iv = invT[H[j + 1][j]];
        for (int i = j + 2; i < m; ++i) {
            if (!H[i][j]) continue;
            const uint32_t f = mul(H[i][j], iv);
            for (int k = 0; k < m; ++k) H[i][k] = (uint8_t)sub(H[i][k], mul(f, H[j + 1][k]));
            for (int k = 0; k < m; ++k) H[k][j + 1] = (uint8_t)add(H[k][j + 1], mul(f, H[k][i]));
        }
    }
    // p_k(t) = (t - h_kk) p_{k-1} - sum_{i<k} h_ik (prod_{j=i+1..k} h_{j,j-1}) p_{i-1}  (1-based)
    uint8_t P[MX + 1][MX + 1];
    P[0][0] = 1;
    for (int k = 1; k <= m; ++k) {
        for (int e = 0; e <= k; ++e) {   // (t - h_kk) p_{k-1}
            uint32_t v = (e >= 1) ? P[k - 1][e - 1] : 0u;
            if (e <= k - 1) v = sub(v, mul(H[k - 1][k - 1], P[k - 1][e]));
            P[k][e] = (uint8_t)v;
        }
        uint32_t prod = 1;
        for (int i = k - 1; i >= 1; --i) {
            prod = mul(prod, H[i][i - 1]);            // h_{i+1,i} (1-based)
            const uint32_t f = mul(H[i - 1][k - 1], prod);
            if (!f) continue;
            for (int e = 0; e <= i - 1; ++e) P[k][e] = (uint8_t)sub(P[k][e], mul(f, P[i - 1][e]));
        }
    }
    // member c square-free iff chi(-c) != 0; chi is monic of degree m
    uint32_t mask = 0;
    for (uint32_t c = 0; c < q; ++c) {
        const uint8_t *mrow = mulT + subT[c] * q;   // times t = -c
        uint32_t v = 1;
        for (int e = m - 1; e >= 0; --e) v = addT[mrow[v] * q + P[m][e]];
        if (v) mask |= 1u << c;
    }
    return mask;
}

// sqf_mask_for_b when f' = w has full degree D - 1 (its leading coefficient
// D c_D is nonzero: p does not divide D): the same steps -- g_b mod w, the
// matrix of multiplication by g_b on F_q[x]/(w), its upper Hessenberg form,
// the Hessenberg recurrence for the characteristic polynomial, its values at
// t = -c -- with every loop bound fixed, so that the matrix and the
// polynomials stay in registers.  A zero subdiagonal pivot is replaced by the
// first nonzero entry below it through a row and column swap made of selects.
template <int D>
__device__ __noinline__ uint32_t sqf_mask_full(const uint8_t *mulT, const uint8_t *subT, const uint8_t *invT,
                                               const uint8_t *addT, uint32_t q, uint32_t p, const uint32_t *cg,
                                               uint32_t b)
{
    constexpr int M = D - 1;   // deg w
    auto mul = [&](uint32_t x, uint32_t y) -> uint32_t { return mulT[x * q + y]; };
    auto sub = [&](uint32_t x, uint32_t y) -> uint32_t { return subT[x * q + y]; };
    auto add = [&](uint32_t x, uint32_t y) -> uint32_t { return addT[x * q + y]; };
    // w = f' / (D c_D), monic
    uint32_t w[M + 1];
    w[0] = b;
#pragma unroll
    for (int i = 2; i <= D; ++i) w[i - 1] = mul((uint32_t)i % p, cg[i]);
    const uint32_t wi = invT[w[M]];
#pragma unroll
    for (int i = 0; i < M; ++i) w[i] = mul(w[i], wi);
    // r = g_b mod w, g_b = b x + sum_{i>=2} c_i x^i
    uint32_t r[D + 1];
    r[0] = 0;
    r[1] = b;
#pragma unroll
    for (int i = 2; i <= D; ++i) r[i] = cg[i];
#pragma unroll
    for (int t = D; t >= M; --t) {
        const uint32_t cf = r[t];
        r[t] = 0;
#pragma unroll
        for (int i = 0; i < M; ++i) r[t - M + i] = sub(r[t - M + i], mul(cf, w[i]));
    }
    // H[i][j]: coefficient i of g_b x^j mod w
    uint32_t H[M][M];
#pragma unroll
    for (int j = 0; j < M; ++j) {
#pragma unroll
        for (int i = 0; i < M; ++i) H[i][j] = r[i];
        if (j + 1 < M) {
            const uint32_t top = r[M - 1];
#pragma unroll
            for (int i = M - 1; i >= 1; --i) r[i] = sub(r[i - 1], mul(top, w[i]));
            r[0] = sub(0, mul(top, w[0]));
        }
    }
    // upper Hessenberg form by similarity
#pragma unroll
    for (int j = 0; j + 2 < M; ++j) {
#pragma unroll
        for (int i = j + 2; i < M; ++i) {
            const bool sw = H[j + 1][j] == 0 && H[i][j] != 0;
#pragma unroll
            for (int k = 0; k < M; ++k) {
                const uint32_t x = H[i][k], y = H[j + 1][k];
                H[i][k] = sw ? y : x;
                H[j + 1][k] = sw ? x : y;
            }
#pragma unroll
            for (int k = 0; k < M; ++k) {
                const uint32_t x = H[k][i], y = H[k][j + 1];
                H[k][i] = sw ? y : x;
                H[k][j + 1] = sw ? x : y;
            }
        }
        // a zero pivot leaves a zero column below it: every f is 0
        const uint32_t iv = invT[H[j + 1][j]];
#pragma unroll
        for (int i = j + 2; i < M; ++i) {
            const uint32_t f = mul(H[i][j], iv);
#pragma unroll
            for (int k = 0; k < M; ++k) H[i][k] = sub(H[i][k], mul(f, H[j + 1][k]));
#pragma unroll
            for (int k = 0; k < M; ++k) H[k][j + 1] = add(H[k][j + 1], mul(f, H[k][i]));
        }
    }
    // p_k(t) = (t - h_kk) p_{k-1} - sum_{i<k} h_ik (prod_{j=i+1..k} h_{j,j-1}) p_{i-1}  (1-based)
    uint32_t P[M + 1][M + 1];
    P[0][0] = 1;
#pragma unroll
    for (int k = 1; k <= M; ++k) {
#pragma unroll
        for (int e = 0; e <= k; ++e) {
            uint32_t v = (e >= 1) ? P[k - 1][e - 1] : 0u;
            if (e <= k - 1) v = sub(v, mul(H[k - 1][k - 1], P[k - 1][e]));
            P[k][e] = v;
        }
        uint32_t prod = 1;
#pragma unroll
        for (int i = k - 1; i >= 1; --i) {
            prod = mul(prod, H[i][i - 1]);
            const uint32_t f = mul(H[i - 1][k - 1], prod);
#pragma unroll
            for (int e = 0; e <= i - 1; ++e) P[k][e] = sub(P[k][e], mul(f, P[i - 1][e]));
        }
    }
    // member c square-free iff chi(-c) != 0
    uint32_t mask = 0;
    for (uint32_t c = 0; c < q; ++c) {
        const uint8_t *mrow = mulT + subT[c] * q;   // times t = -c
        uint32_t v = 1;
#pragma unroll
        for (int e = M - 1; e >= 0; --e) v = addT[mrow[v] * q + P[M][e]];
        if (v) mask |= 1u << c;
    }
    return mask;
}

// one group of q^2 members (c_1, c_0 free) for one warp.  W: a sampled
// family counted over its whole family, each member with its multiplicity
// among the samples (KJob::mweight; a separate instantiation, so that the
// unweighted code stays as it is)
template <int D, bool W>
__device__ __forceinline__ void process_group2(const KJob &J, uint64_t gtile, const uint8_t *smem,
                                               uint8_t *wsm, int lane, WarpStats &st)
{
    constexpr int G = (D - 1) / 2;
    const uint32_t q = J.q, qq = q * q;
    const uint64_t base = (J.first_group + gtile) * qq;
    uint32_t c[D + 1];
    decode_index<D>(J, base, c);
    c[0] = 0;
    c[1] = 0;
    uint32_t nz = 0;
#pragma unroll
    for (int i = 2; i < D; ++i) nz |= (c[i] != 0 ? 1u : 0u) << i;

    // per-warp shared scratch (fan2_layout); the members' keys live in this
    // warp's slot of global scratch
    const Fan2Layout lay = fan2_layout(q, J.dense_off != 0);
    uint16_t *a1s = reinterpret_cast<uint16_t *>(wsm + lay.a1_off);   // dense histogram: a_1 + 32768
    uint32_t *dense = reinterpret_cast<uint32_t *>(const_cast<uint8_t *>(smem) + J.dense_off);
    uint32_t *Us = reinterpret_cast<uint32_t *>(wsm);
    uint32_t *Ds = reinterpret_cast<uint32_t *>(wsm + lay.ds_off);
    uint16_t *acc = reinterpret_cast<uint16_t *>(wsm + lay.acc_off);
    uint16_t *rq = reinterpret_cast<uint16_t *>(wsm + lay.rq_off);
    uint32_t *sqfw = reinterpret_cast<uint32_t *>(wsm + lay.sqf_off);
    uint32_t *gc = reinterpret_cast<uint32_t *>(wsm + lay.par_off);   // c_0..c_D
    uint32_t *glam = gc + 12;                                          // lam_0..lam_D of the field
    HChain<D> *gH = reinterpret_cast<HChain<D> *>(gc + 24);
    static_assert(sizeof(HChain<D>) <= 4 * (64 - 24), "h chain exceeds the warp's parameter block");
    const uint32_t nw = (qq + 31) / 32;
    unsigned long long *keys =
        J.wkeys + ((uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * J.wkeys_stride;

    const uint32_t *s32 = reinterpret_cast<const uint32_t *>(smem);
    const uint8_t *mulT = smem + J.fq_off;
    const uint8_t *subT = mulT + qq;
    const uint8_t *invT = subT + qq;
    const uint8_t *addT = invT + q;

    // square-freeness: lane b settles the q members with c_1 = b at once
    for (uint32_t t = lane; t < nw; t += 32) sqfw[t] = 0;
    if (64 + (uint32_t)lane < lay.us) {   // slack read by 8-point blocks past 64
        Us[64 + lane] = 0;
        Ds[64 + lane] = 0;
    }
    if (lane == 0) {
#pragma unroll
        for (int i = 0; i <= D; ++i) gc[i] = c[i];
    }
    __syncwarp();
    if ((uint32_t)lane < q) {
        uint32_t mask;
        if constexpr (D <= 10) {   // f' of full degree: the fixed-shape form
            if (mulT[(D % J.p) * q + gc[D]] != 0) mask = sqf_mask_full<D>(mulT, subT, invT, addT, q, J.p, gc, (uint32_t)lane);
            else mask = sqf_mask_for_b<D>(mulT, subT, invT, addT, q, J.p, gc, (uint32_t)lane);
        } else {
            mask = sqf_mask_for_b<D>(mulT, subT, invT, addT, q, J.p, gc, (uint32_t)lane);
        }
        // bits b*q .. b*q + q-1 of the member mask
        const uint32_t bit0 = (uint32_t)lane * q;
        const uint32_t w0 = bit0 >> 5, sh = bit0 & 31u;
        if (mask) {
            atomicOr(&sqfw[w0], mask << sh);
            if (sh && sh + q > 32) atomicOr(&sqfw[w0 + 1], mask >> (32 - sh));
        }
    }
    __syncwarp();
    uint32_t anyv = 0, anys = 0;
    if constexpr (W) {
        for (uint32_t t = 0; t < nw; ++t) {
            const uint32_t m = t * 32 + lane;
            const uint64_t idx = base + m;
            bool v = m < qq && idx >= J.first && idx < J.first + J.count;
            const uint32_t w = v ? J.mweight[idx - J.w_first] : 0u;   // multiplicity among the samples (0: not drawn)
            v = v && w != 0;
            const bool sq = v && ((sqfw[t] >> lane) & 1u);
            const unsigned vm = __ballot_sync(0xFFFFFFFFu, v);
            const unsigned sm = __ballot_sync(0xFFFFFFFFu, sq);
            const uint32_t wv = __reduce_add_sync(0xFFFFFFFFu, v ? w : 0u);
            const uint32_t ws = __reduce_add_sync(0xFFFFFFFFu, sq ? w : 0u);
            __syncwarp();
            if (lane == 0) {
                sqfw[t] = sm;   // square-free, in range and drawn
                st.examined += wv;
                st.sqf += ws;
            }
            anyv |= vm;
            anys |= sm;
        }
    } else {
        for (uint32_t t = 0; t < nw; ++t) {
            const uint32_t m = t * 32 + lane;
            const uint64_t idx = base + m;
            const bool v = m < qq && idx >= J.first && idx < J.first + J.count;
            const bool sq = v && ((sqfw[t] >> lane) & 1u);
            const unsigned vm = __ballot_sync(0xFFFFFFFFu, v);
            const unsigned sm = __ballot_sync(0xFFFFFFFFu, sq);
            __syncwarp();
            if (lane == 0) {
                sqfw[t] = sm;   // square-free and in range
                st.examined += __popc(vm);
                st.sqf += __popc(sm);
            }
            anyv |= vm;
            anys |= sm;
        }
    }
    __syncwarp();
    if ((J.unfiltered ? anyv : anys) == 0) {
        if (J.member_counts) {
            for (uint32_t m = lane; m < qq; m += 32) {
                const uint64_t idx = base + m;
                if (idx < J.first || idx >= J.first + J.count) continue;
#pragma unroll
                for (int k = 0; k < G; ++k) J.member_counts[(idx - J.first) * G + k] = 0;
                J.member_sqf[idx - J.first] = 0;
            }
        }
        return;
    }

    // lane roles: S lanes per value b of c_1, each taking a chunk of the points;
    // lane = s q + b owns accumulator row `lane`
    const uint32_t S = 32 / q;
    const bool role = (uint32_t)lane < S * q;
    const uint32_t b = role ? (uint32_t)lane % q : 0;
    const uint32_t s = role ? (uint32_t)lane / q : 0;
    uint16_t *acc_row = acc + (uint32_t)lane * q;   // lanes past S q: rows no member reads
    const uint32_t acc_words = 16 * q;
    // one point per Frobenius orbit: S_k = sum_{m | k} m (E_m or N_m - Z_m)
    // (orbit_combine); each member's partial sums of the later S_k wait in its
    // key slots (or, with the dense box, next to a_1)
    const bool orb = G >= 2 && J.reps[G >= 2 ? 1 : 0] != nullptr;

#pragma unroll 1
    for (int k = 0; k < G; ++k) {
        const uint32_t L = J.L[k], Q = J.Q[k];
        const uint32_t *coefk = s32 + J.coef_off[k];
        if (lane == 0) {
            uint32_t lam[D + 1];
#pragma unroll
            for (int i = 0; i <= D; ++i) lam[i] = coefk[gc[i]];
            HChain<D> H;
            make_hchain<D, 2>(H, lam, nz, L);
            *gH = H;
#pragma unroll
            for (int i = 0; i <= D; ++i) glam[i] = lam[i];
        }
        for (uint32_t m = lane; m < acc_words; m += 32) reinterpret_cast<uint32_t *>(acc)[m] = 0;
        __syncwarp();
        const bool tri = J.tab_kind[k] == kTabTripleSmem;
        const uint32_t zs = J.zshift[k];
        const uint32_t zw = zs ? 1u + (1u << zs) : 1u;
        // zero digits: counted directly in F_q and F_{q^2} (with its coordinates)
        // when g <= 2; queued for g >= 3, whose time is in F_{q^3} and up (one
        // copy of the field loop for every field keeps the instruction cache warm)
        // (degrees 2g+1, 2g+2 >= 7 are g >= 3: no direct copies compiled)
        const int kf = J.g > 2 ? 0 : (k == 0 ? 1 : (J.coord_off ? 2 : 0));
        if constexpr (D <= 6) {
            if (kf == 1) group2_field_tabs<D, 1>(J, k, tri, smem, gH, glam, nz, Us, Ds, acc, acc_row, rq, lane, role, b, s, S, zw);
            else if (kf == 2) group2_field_tabs<D, 2>(J, k, tri, smem, gH, glam, nz, Us, Ds, acc, acc_row, rq, lane, role, b, s, S, zw);
            else group2_field_tabs<D, 0>(J, k, tri, smem, gH, glam, nz, Us, Ds, acc, acc_row, rq, lane, role, b, s, S, zw);
        } else {
            (void)kf;
            group2_field_tabs<D, 0>(J, k, tri, smem, gH, glam, nz, Us, Ds, acc, acc_row, rq, lane, role, b, s, S, zw);
        }
        __syncwarp();
        // over the field's points: sum chi(f_{b,c}) = (points - (2 cnt + z)) + chi(c) for x = 0,
        // which belongs to F_q (and to every field when every point is evaluated)
        int inf = 1;
        if (D == 2 * G + 2) inf += (glam[D] & 1u) ? -1 : 1;
        const bool x0 = J.reps[k] == nullptr;
        const int npts = (int)J.npts[k];
        const int Nm = npts + (x0 ? 1 : 0);
        if ((uint32_t)lane < q) {
            const uint32_t cc = (uint32_t)lane;
            const uint32_t lc = coefk[cc];
            const int chi_c = (cc == 0) ? 0 : ((lc & 1u) ? -1 : 1);
            // the members' key slots (global scratch) from the earlier fields,
            // loaded one member ahead
            const bool keyed = !J.dense_off && k > 0;
            unsigned long long knext = keyed ? keys[cc] : 0ull;
            for (uint32_t bb = 0; bb < q; ++bb) {
                const uint32_t m = bb * q + cc;
                const unsigned long long kold = knext;
                if (keyed && bb + 1 < q) knext = keys[m + q];
                uint32_t tot = 0;
                for (uint32_t ss = 0; ss < S; ++ss) tot += acc[(ss * q + bb) * q + cc];
                const int a2 = zs ? (int)(tot & ((1u << zs) - 1u)) : (int)tot;
                const int E = npts - a2 + (x0 ? chi_c : 0);
                const int Z = (zs ? (int)(tot >> zs) : 0) + ((x0 && cc == 0) ? 1 : 0);
                // partial sum of S_{k+1} from the smaller fields, then this field's share
                int Sk = E;
                if (orb) {
                    int part = 0;
                    if (J.dense_off) part = k == 1 ? (int)(a1s[m] >> 8) : 0;
                    else if (k > 0) part = (int16_t)(uint16_t)(kold >> (16 * k));
                    Sk = part + (k + 1) * E;
                }
                const int N = (int)Q + Sk + inf;
                if (J.member_counts) {
                    const uint64_t idx = base + m;
                    if (idx >= J.first && idx < J.first + J.count) {
                        const bool sq = (sqfw[m / 32] >> (m % 32)) & 1u;
                        J.member_counts[(idx - J.first) * G + k] = (sq || J.unfiltered) ? N : 0;
                        if (k == 0) J.member_sqf[idx - J.first] = sq ? 1 : 0;
                    }
                }
                const int a = (int)Q + 1 - N;   // eq. 1.1
                const uint32_t a16 = (uint32_t)(a + 32768) & 0xFFFFu;
                if (J.dense_off) {
                    // g <= 2: a_1 (and, with orbits, the field-1 part N_1 - Z_1 of S_2)
                    // wait in shared memory; the last field counts the member
                    if (k + 1 < G) {
                        a1s[m] = (uint16_t)(((uint32_t)(a + 128) & 0xFFu) | (orb ? (uint32_t)(Nm - Z) << 8 : 0u));
                    } else if (!J.member_counts && ((sqfw[m / 32] >> (m % 32)) & 1u)) {
                        const uint32_t k1 = G == 2 ? ((a1s[m] & 0xFFu) + 32768u - 128u) : a16;
                        const int i1 = (int)k1 - 32768 + J.dense_b1;
                        const int i2 = G == 2 ? a + J.dense_b2 : 0;
                        uint32_t w = 1;
                        if constexpr (W) w = J.mweight[base + m - J.w_first];
                        if (i1 >= 0 && i1 <= 2 * J.dense_b1 && i2 >= 0 && i2 <= 2 * J.dense_b2)
                            atomicAdd(&dense[(uint32_t)i1 * J.dense_w2 + (uint32_t)i2], w);
                        else   // outside the Hasse-Weil box: not for a smooth curve
                            hist_insert(J, G == 2 ? ((unsigned long long)a16 << 16 | k1) : a16, w);
                    }
                } else {
                    // slot k: this member's final a_{k+1}; with orbits, slots of the
                    // multiples (k+1) t collect (k+1) (E or N - Z) as int16
                    unsigned long long key = k == 0 ? 0ull : kold;
                    key = (key & ~(0xFFFFull << (16 * k))) | ((unsigned long long)a16 << (16 * k));
                    if (orb) {
#pragma unroll
                        for (int t = 2; t <= G; ++t) {
                            const int kk = (k + 1) * t - 1;
                            if (kk >= G) break;
                            const int add = (k + 1) * ((t & 1) ? E : Nm - Z);
                            const int cur = k == 0 ? 0 : (int)(int16_t)(uint16_t)(key >> (16 * kk));
                            key = (key & ~(0xFFFFull << (16 * kk))) |
                                  ((unsigned long long)(uint16_t)(int16_t)(cur + add) << (16 * kk));
                        }
                    }
                    keys[m] = key;
                }
            }
        }
        __syncwarp();
    }
    if (J.member_counts || J.dense_off) return;   // dense: counted with the last field
    __syncwarp();
    for (uint32_t t = 0; t < nw; ++t) {
        const uint32_t m = t * 32 + lane;
        const bool sq = m < qq && ((sqfw[t] >> lane) & 1u);
        const unsigned smask = __ballot_sync(0xFFFFFFFFu, sq);
        if (sq) {
            const unsigned long long key = keys[m];
            const unsigned peers = __match_any_sync(smask, key);
            // equal keys counted once: the peers' members, or their multiplicities
            uint32_t cnt;
            if constexpr (W) cnt = __reduce_add_sync(peers, J.mweight[base + m - J.w_first]);
            else cnt = __popc(peers);
            if (lane == __ffs(peers) - 1) hist_insert(J, key, cnt);
        }
    }
    __syncwarp();
}

// the CTA's dense (a_1, a_2) counters into the job's histogram (all threads;
// the counters must be complete: call after a barrier)
__device__ void flush_dense(const KJob &J, const uint8_t *smem)
{
    const uint32_t *dense = reinterpret_cast<const uint32_t *>(smem + J.dense_off);
    for (uint32_t i = threadIdx.x; i < J.dense_n; i += blockDim.x) {
        const uint32_t c = dense[i];
        if (!c) continue;
        const int a1 = (int)(i / J.dense_w2) - J.dense_b1;
        const int a2 = (int)(i % J.dense_w2) - J.dense_b2;
        unsigned long long key = (unsigned long long)((uint32_t)(a1 + 32768) & 0xFFFFu);
        if (J.g == 2) key |= (unsigned long long)((uint32_t)(a2 + 32768) & 0xFFFFu) << 16;
        hist_insert(J, key, c);
    }
}

// threads per CTA at most: 24 warps at <= 80 registers for degrees <= 6, 16
// warps above (whose longer coefficient arrays would spill at 80)
template <int D, bool W>
__global__ void __launch_bounds__(D <= 6 ? 768 : 512, 1)
    k_fan2_persistent(const KJob *__restrict__ jobs, const uint64_t *__restrict__ item_start, uint32_t n_jobs,
                      uint64_t n_items, unsigned long long *counter, uint32_t item_tiles)
{
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ unsigned long long s_item;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwp = blockDim.x >> 5;
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
            if (cur >= 0) {
                flush_stats(jobs[cur], st, lane);
                if (jobs[cur].dense_off) flush_dense(jobs[cur], smem);
                __syncthreads();
            }
            stage_job(jobs[jb], smem);
            __syncthreads();
            cur = jb;
        }
        const KJob &J = jobs[jb];
        uint8_t *wsm = smem + J.warp_off + warp * J.warp_bytes;
        const uint64_t t0 = (item - item_start[jb]) * item_tiles;
        const uint64_t t1 = min(t0 + item_tiles, J.n_tiles);
        for (uint64_t t = t0 + warp; t < t1; t += nwp) process_group2<D, W>(J, t, smem, wsm, lane, st);
        __syncthreads();
    }
    if (cur >= 0) {
        flush_stats(jobs[cur], st, lane);
        if (jobs[cur].dense_off) flush_dense(jobs[cur], smem);
    }
}

template <int D, bool W = false>
const void *fan2_pick()
{
    return (const void *)k_fan2_persistent<D, W>;
}

}  // namespace
}  // namespace hwc
