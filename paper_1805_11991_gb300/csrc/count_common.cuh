// count_common.cuh -- device pieces shared by the count kernels: table
// access, member decoding, the square-free test, Zech chain steps and the
// histogram hash.  Included by count_kernels.cu and fanout_kernels.cu only.
#pragma once
#include "hwc_internal.cuh"

namespace hwc {
namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;

struct TabS {   // u16 table in shared memory
    const uint16_t *t;
    __device__ __forceinline__ uint32_t operator[](uint32_t u) const { return t[u]; }
};
template <bool PAD>
struct TabP {   // staged two-level Zech table: index u at u + 64; PAD: entry i at i + 2 floor(i / 64)
    const uint16_t *t;
    __device__ __forceinline__ uint32_t at(uint32_t i) const { return PAD ? t[i + ((i >> 6) << 1)] : t[i]; }
    __device__ __forceinline__ uint32_t operator[](uint32_t u) const { return at(u + kFan2Prefix); }
};
// 17-bit Zech table in shared memory (fields whose logs exceed 16 bits): the
// low 16 bits of entry v in lo[v], bit 16 in bit v of the plane hi.  Read with
// the doubled index range of TabS / TabG: u in [0, 2L] folds to v in [0, L] by
// one subtraction; entries L/2 and L hold the marker 0x1FFFF, returned as the
// poison 2L.
struct Tab17 {
    const uint16_t *lo;
    const uint32_t *hi;
    uint32_t L;
    __device__ __forceinline__ uint32_t operator[](uint32_t u) const
    {
        const uint32_t v = min(u, u - L);
        const uint32_t w = (uint32_t)lo[v] | (((hi[v >> 5] >> (v & 31u)) & 1u) << 16);
        return w == 0x1FFFFu ? 2 * L : w;
    }
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
// member decoding (the choice of f in Algorithm 1; family definitions in hwc.h)

// member idx of the reduced family (HWC_FAM_REDUCED): pattern by its start
// index, then the digits; returns the pattern
template <int D>
__device__ __forceinline__ uint32_t decode_reduced(const KJob &J, uint64_t idx, uint32_t (&c)[D + 1])
{
    uint32_t pt = 0;
    while (pt + 1 < J.red_n && J.red_start[pt + 1] <= idx) ++pt;
    uint64_t r = idx - J.red_start[pt];
    const uint32_t q = J.q;
#pragma unroll
    for (int i = 0; i <= D; ++i) c[i] = 0;
    const uint32_t pi = J.red_i[pt], pj = J.red_j[pt];
    if (pi >= 0xFE) {   // A: c_d X^d + 1, B: c_d X^d + X
        c[D] = 1 + (uint32_t)r;
        if (pi == 0xFF) c[0] = 1;
        else c[1] = 1;
        return pt;
    }
#pragma unroll
    for (int i = 0; i < D; ++i)
        if ((uint32_t)i < pj) {
            c[i] = (uint32_t)(r % q);
            r /= q;
        }
    const uint32_t gg = J.red_gcd[pt];
    const uint32_t t = (uint32_t)(r % gg);
    c[D] = 1 + (uint32_t)(r / gg);
    const uint32_t w = J.red_w[t];
#pragma unroll
    for (int i = 0; i < D; ++i) {   // static indices: c stays in registers
        if ((uint32_t)i == pi) c[i] = 1;
        if ((uint32_t)i == pj) c[i] = w;
    }
    return pt;
}

template <int D>
__device__ __forceinline__ void decode_member(const KJob &J, uint64_t m, uint32_t (&c)[D + 1])
{
    uint64_t idx = J.first + m;
    uint32_t kind = J.kind;
    if (kind == HWC_FAM_REDUCED) {
        decode_reduced<D>(J, idx, c);
        return;
    }
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

// Quadratic character of the discriminant of a square-free f over F_q (logs of
// the coefficients as in squarefree(); f' is taken with its true degree e):
//     disc f = (-1)^(d(d-1)/2) lc(f)^(-1) Res_{d,d-1}(f, f'),
//     Res_{d,d-1}(f, f') = lc(f)^(d-1-e) Res_{d,e}(f, f'),
// and Res_{d,e} by Euclid's algorithm, Res(A, B) = (-1)^(ab) lc(B)^(a-r) Res(B, A mod B)
// (r = deg(A mod B)), Res(A, c) = c^a for a constant c.  chi of a product is
// the product of the chi: the parity of the logs, and chi(-1) = (-1)^((q-1)/2).
// Returns +1 or -1.
template <int D, class Tab>
__device__ int disc_chi(const FqLog<Tab> &F, const uint32_t *coef1, uint32_t p, uint32_t q,
                        const uint32_t (&c)[D + 1])
{
    const uint32_t Z = F.L;
    const uint32_t neg1 = ((q - 1) / 2) & 1u;   // parity of chi(-1)
    uint32_t P[2][D + 1];
    int dg[2];
    for (int i = 0; i <= D; ++i) P[0][i] = coef1[c[i]];
    for (int i = 1; i <= D; ++i) P[1][i - 1] = F.mul(coef1[i % p], P[0][i]);
    P[1][D] = Z;
    dg[0] = D;
    dg[1] = D - 1;
    while (dg[0] >= 0 && P[0][dg[0]] == Z) --dg[0];
    while (dg[1] >= 0 && P[1][dg[1]] == Z) --dg[1];
    const int d = dg[0], e = dg[1];
    // (-1)^(d(d-1)/2) lc(f)^(-1) lc(f)^(d-1-e): parity of the log of lc(f) counts d - e times
    uint32_t par = (((uint32_t)(d * (d - 1) / 2)) & 1u) * neg1;
    par ^= (P[0][d] & 1u) * ((uint32_t)(d - e) & 1u);
    int a = 0, b = 1;
    for (;;) {
        const int da = dg[a], db = dg[b];
        if (db == 0) {   // Res(A, c) = c^a
            par ^= (P[b][0] & 1u) * ((uint32_t)da & 1u);
            break;
        }
        const uint32_t lb = P[b][db];
        const uint32_t il = (F.L - lb) % F.L;
        for (int t = da; t >= db; --t) {
            if (P[a][t] == Z) continue;
            const uint32_t cf = F.mul(P[a][t], il);
            for (int i = 0; i <= db; ++i) P[a][t - db + i] = F.add(P[a][t - db + i], F.neg(F.mul(cf, P[b][i])));
        }
        int dr = db - 1;
        while (dr >= 0 && P[a][dr] == Z) --dr;
        // f square-free: the remainder sequence ends in a nonzero constant
        par ^= (((uint32_t)(da * db)) & 1u) * neg1;
        par ^= (lb & 1u) * ((uint32_t)(da - dr) & 1u);
        dg[a] = dr;
        const int tmp = a;
        a = b;
        b = tmp;
    }
    return par ? -1 : 1;
}

// ---------------------------------------------------------------------
// one field: sum over x in F_Q^x of chi(f(x)) for this lane's share of x
//
// Two table layouts: TRIPLE (entries over [0, 3L], poison 3L) lets a step be
// u <- min(T[u] + d + g*j, 3L) with d, g*j < L and no reduction; DOUBLE
// (entries over [0, 2L], poison 2L) reduces d + g*j mod L first.

// Horner in the log domain with explicit zero handling, for the rare x at
// which some partial sum vanishes (the chain above then holds the poison).
template <int D, class Tab>
__device__ __forceinline__ int slow_chi(const Tab T, uint32_t L, uint32_t cap,
                                        const uint32_t (&lam)[D + 1], uint32_t nz, uint32_t j)
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
                const uint32_t n = addmod(l, L - lam[i], L);
                const uint32_t z = T[n];
                if (z >= cap) zero = true;
                else l = addmod(lam[i], z, L);
            }
        }
    }
    return zero ? 0 : ((l & 1u) ? -1 : 1);
}

template <bool TRIPLE>
__device__ __forceinline__ uint32_t chain_step(uint32_t z, uint32_t d, uint32_t m, uint32_t L, uint32_t cap)
{
    if (TRIPLE) return min(z + d + m, cap);
    return min(z + addmod(d, m, L), cap);
}

// dense chain: every coefficient below position I1 is nonzero (all gaps 1)
// ---------------------------------------------------------------------
// histogram

__device__ __forceinline__ void hist_insert(const KJob &J, unsigned long long key, unsigned long long cnt)
{
    uint32_t h = (uint32_t)mix64(key) & J.hmask;
    for (uint32_t probe = 0; probe <= J.hmask; ++probe) {
        unsigned long long cur = *((volatile unsigned long long *)&J.hkeys[h]);
        if (cur == kEmptyKey) cur = atomicCAS(&J.hkeys[h], kEmptyKey, key);
        if (cur == kEmptyKey || cur == key) {
            atomicAdd(&J.hcounts[h], cnt);
            return;
        }
        h = (h + 1) & J.hmask;
    }
    atomicOr(&J.stats[2], 1ull);   // table full
}

struct WarpStats {
    uint32_t examined = 0;   // members in range (weighted by their draws for sampled families, < 2^27)
    unsigned long long sqf = 0;   // square-free members (weighted for reduced families)
};

// S_k = sum over x in F_{q^k} of chi_{q^k}(f(x)) from the sums of the fields'
// points.  With one point per Frobenius orbit (J.reps[1] set): chi(f(x)) is
// constant on the orbit {x, x^q, ...} (f has coefficients in F_q), an element
// of exact degree m has m conjugates, and chi_{q^k}(y) = chi_{q^m}(y)^(k/m) for
// y in F_{q^m}, so
//     S_k = sum_{m | k} m * (E_m if k/m is odd, else N_m - Z_m),
// E_m = sum of chi_{q^m}(f(x)), Z_m = number of zeros of f, N_m = number of
// points, over the orbit points of exact degree m (x = 0 belongs to m = 1).
// Every point evaluated (J.reps[1] null): S_k = E_k.
template <int G>
__device__ __forceinline__ void orbit_combine(const KJob &J, const int (&E)[G], const int (&Z)[G], int (&S)[G])
{
    const bool orb = G >= 2 && J.reps[G >= 2 ? 1 : 0] != nullptr;
#pragma unroll
    for (int k = 1; k <= G; ++k) {
        if (!orb) {
            S[k - 1] = E[k - 1];
            continue;
        }
        int s = 0;
#pragma unroll
        for (int m = 1; m <= k; ++m) {
            if (k % m) continue;
            const int Nm = m == 1 ? (int)J.q : (int)J.npts[m - 1];
            s += m * (((k / m) & 1) ? E[m - 1] : Nm - Z[m - 1]);
        }
        S[k - 1] = s;
    }
}

// copy the job's tables into shared memory (all threads of the CTA)
__device__ void stage_job(const KJob &J, uint8_t *smem)
{
    uint16_t *s16 = reinterpret_cast<uint16_t *>(smem);
    uint32_t *s32 = reinterpret_cast<uint32_t *>(smem);
    for (uint32_t k = 0; k < J.g; ++k) {
        if (J.tab_kind[k] == kTab17Smem) {   // low halves, then the plane of high bits
            uint16_t *dst = s16 + J.tab_off[k];
            for (uint32_t i = threadIdx.x; i <= J.L[k]; i += blockDim.x) dst[i] = J.z17lo[k][i];
            uint32_t *dhi = reinterpret_cast<uint32_t *>(s16 + J.tab_hi_off[k]);
            for (uint32_t i = threadIdx.x; i < (J.L[k] + 32) / 32; i += blockDim.x) dhi[i] = J.z17hi[k][i];
        } else if (J.tab_kind[k] != kTabDoubleGlobal) {
            const bool tri = J.tab_kind[k] == kTabTripleSmem;
            const uint32_t n = (tri ? 3 : 2) * J.L[k] + 1;
            const uint16_t *src = tri ? J.zech3[k] : J.zech2[k];
            uint16_t *dst = s16 + J.tab_off[k];
            if (J.method == 2) {   // periodic prefix, poison 0xFFFF, optional pad word per 32
                const int Li = (int)J.L[k];
                for (uint32_t i = threadIdx.x; i < n + kFan2Prefix; i += blockDim.x) {
                    const int u = (int)i - (int)kFan2Prefix;
                    uint32_t v = src[u >= 0 ? u : ((u % Li) + Li) % Li];
                    if (v >= J.L[k]) v = 0xFFFFu;
                    dst[J.tab_pad[k] ? i + ((i >> 6) << 1) : i] = (uint16_t)v;
                }
            } else {
                for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
            }
        }
        const uint32_t *src = J.coef_log[k];
        uint32_t *dst = s32 + J.coef_off[k];
        for (uint32_t i = threadIdx.x; i < J.q; i += blockDim.x) dst[i] = src[i];
        if (J.method != 0) {
            const uint32_t L = J.L[k];
            const uint32_t *rs = reinterpret_cast<const uint32_t *>(J.rows[k]);
            uint32_t *rd = reinterpret_cast<uint32_t *>(smem + J.row_off[k]);
            if (J.method == 2 && J.row16[k]) {   // int16 rows: q <= 15 digit bits, the flag (bit 31) in bit 15
                int16_t *rd16 = reinterpret_cast<int16_t *>(rd);
                for (uint32_t i = threadIdx.x; i <= L + kFan2ZeroRow; i += blockDim.x) {
                    const uint32_t v = rs[i < L ? i : (i < L + kFan2ZeroRow ? (i - L) % L : L)];
                    rd16[i] = (int16_t)(uint16_t)((v & 0x7FFFu) | ((v >> 16) & 0x8000u));
                }
            } else if (J.method == 2) {   // rows[i mod L] for i < L + 8, then y = 0 (row L of the table)
                for (uint32_t i = threadIdx.x; i <= L + kFan2ZeroRow; i += blockDim.x)
                    rd[i] = rs[i < L ? i : (i < L + kFan2ZeroRow ? (i - L) % L : L)];
            } else {
                const uint32_t nw = (L + 1) * J.words;   // row L: y = 0
                for (uint32_t i = threadIdx.x; i < nw; i += blockDim.x) rd[i] = rs[i];
            }
            uint8_t *zd = smem + J.zdig_off[k];
            for (uint32_t i = threadIdx.x; i < J.q; i += blockDim.x) zd[i] = J.zdig[k][i];
        }
    }
    if (J.dense_off) {   // the CTA's dense (a_1, a_2) counters start at zero
        uint32_t *dn = reinterpret_cast<uint32_t *>(smem + J.dense_off);
        for (uint32_t i = threadIdx.x; i < J.dense_n; i += blockDim.x) dn[i] = 0;
    }
    if (J.method != 0) {   // F_q digit arithmetic: mul | sub | inv | add
        const uint32_t qq = J.q * J.q;
        uint8_t *d = smem + J.fq_off;
        for (uint32_t i = threadIdx.x; i < qq; i += blockDim.x) {
            d[i] = J.fq_mul[i];
            d[qq + i] = J.fq_sub[i];
            // x + y = x - (0 - y)
            d[2 * qq + J.q + i] = J.fq_sub[(i / J.q) * J.q + J.fq_sub[i % J.q]];
        }
        for (uint32_t i = threadIdx.x; i < J.q; i += blockDim.x) d[2 * qq + i] = J.fq_inv[i];
    }
    if (J.coord_off) {   // coordinates of F_{q^2} over F_q (two-level kernel)
        uint32_t *d = reinterpret_cast<uint32_t *>(smem + J.coord_off);
        for (uint32_t i = threadIdx.x; i < J.L[1]; i += blockDim.x) d[i] = J.coord2[i];
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

}  // namespace
}  // namespace hwc
