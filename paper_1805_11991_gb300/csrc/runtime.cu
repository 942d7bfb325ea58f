// runtime.cu -- host side of libhwc: jobs, batches (plain / persistent / CUDA
// graph), histograms and the per-member checking path.
#include "hwc_internal.cuh"

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <numeric>

namespace hwc {

static thread_local std::string g_err;

int set_error(int code, const char *fmt, ...)
{
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

// ---------------------------------------------------------------------
// job validation

static bool mul_ok(uint64_t a, uint64_t b, uint64_t *out)
{
    if (a && b > ~0ull / a) return false;
    *out = a * b;
    return true;
}

static bool upow(uint64_t b, uint32_t e, uint64_t *out)
{
    uint64_t r = 1;
    for (uint32_t i = 0; i < e; ++i)
        if (!mul_ok(r, b, &r)) return false;
    *out = r;
    return true;
}

static int family_size(uint32_t q, const hwc_family_t *fam, uint64_t *n)
{
    uint32_t p, e;
    if (!fam) return set_error(HWC_ERR_ARG, "family is NULL");
    if (!prime_power(q, &p, &e)) return set_error(HWC_ERR_ARG, "q=%u is not an odd prime power", q);
    const uint32_t d = fam->degree;
    if (d < 3 || d > (uint32_t)kMaxD) return set_error(HWC_ERR_ARG, "degree %u outside [3,%d]", d, kMaxD);
    uint64_t v;
    switch (fam->kind) {
    case HWC_FAM_ALL_DEG:
        if (!upow(q, d, &v) || !mul_ok(v, q - 1, &v)) return set_error(HWC_ERR_TOO_LARGE, "family size overflows");
        break;
    case HWC_FAM_MONIC_NOSUB:
        if (!upow(q, d - 1, &v)) return set_error(HWC_ERR_TOO_LARGE, "family size overflows");
        break;
    case HWC_FAM_MONIC_NOSUB_SAMPLED:
        if (!upow(q, d - 1, &v)) return set_error(HWC_ERR_TOO_LARGE, "family size overflows");
        v = fam->sample_count;
        break;
    case HWC_FAM_MONIC_NOSUB_SAMPLED_WINDOW:   // windows name members of the enumerated family
        if (!upow(q, d - 1, &v)) return set_error(HWC_ERR_TOO_LARGE, "family size overflows");
        if (fam->sample_count == 0) return set_error(HWC_ERR_ARG, "windowed sampled family without samples");
        break;
    case HWC_FAM_REDUCED: {   // patterns A, B and (i, j) of Sec. 1.2 (see hwc.h)
        if (d % p == 0) return set_error(HWC_ERR_ARG, "reduced family needs p=%u not dividing d=%u", p, d);
        v = 2ull * (q - 1);
        for (uint32_t i = 1; i + 2 <= d; ++i)
            for (uint32_t j = 0; j < i; ++j) {
                uint64_t t;
                if (!upow(q, j, &t) || !mul_ok(t, (uint64_t)(q - 1) * std::gcd(q - 1, i - j), &t) || v + t < v)
                    return set_error(HWC_ERR_TOO_LARGE, "family size overflows");
                v += t;
            }
        break;
    }
    default:
        return set_error(HWC_ERR_ARG, "unknown family kind %u", fam->kind);
    }
    *n = v;
    return HWC_OK;
}

static int validate_job(const hwc_job_t &j, uint64_t *fam_n)
{
    if (j.g < 1 || j.g > (uint32_t)kMaxG) return set_error(HWC_ERR_ARG, "g=%u outside [1,%d]", j.g, kMaxG);
    const uint32_t d = j.family.degree;
    if (d != 2 * j.g + 1 && d != 2 * j.g + 2)
        return set_error(HWC_ERR_ARG, "degree %u is not 2g+1 or 2g+2 for g=%u", d, j.g);
    int rc = family_size(j.q, &j.family, fam_n);
    if (rc) return rc;
    uint64_t Qg;
    if (!upow(j.q, j.g, &Qg) || Qg > HWC_MAX_Q)
        return set_error(HWC_ERR_TOO_LARGE, "q^g above %u", HWC_MAX_Q);
    if (j.first > *fam_n || j.count > *fam_n - j.first)
        return set_error(HWC_ERR_RANGE, "members [%llu, +%llu) outside the family of %llu",
                         (unsigned long long)j.first, (unsigned long long)j.count,
                         (unsigned long long)*fam_n);
    return HWC_OK;
}

// ---------------------------------------------------------------------
// shared-memory layout of one job: u16 Zech tables first, then u32 coef logs

// Shared-memory layout of one job: u16 Zech tables, u32 digit logs and, for
// the fan-out method, the fan-out rows (4 or 8 bytes each) and zdig bytes.
// Starts from the fastest layout per field (tripled Zech table in smem) and
// moves the largest tables to cheaper-in-space layouts until the job fits.
// Returns false if a fan-out job cannot keep its rows in shared memory.
static uint64_t isqrt_u64(uint64_t v)   // floor(sqrt(v))
{
    uint64_t x = (uint64_t)std::sqrt((double)v);
    while (x * x > v) --x;
    while ((x + 1) * (x + 1) <= v) ++x;
    return x;
}

bool layout_job_smem(KJob &j, uint32_t smem_limit, bool no_triple)
{
    uint32_t kind[kMaxG];
    // the per-member kernel can also read a 17-bit table from shared memory
    auto small17 = [&](uint32_t k) { return j.method == 0 && j.z17lo[k] && j.z17hi[k]; };
    for (uint32_t k = 0; k < j.g; ++k)
        kind[k] = (j.zech3[k] && !no_triple) ? kTabTripleSmem
                  : j.zech2[k]              ? kTabDoubleSmem
                  : small17(k)              ? kTab17Smem
                                            : kTabDoubleGlobal;
    // the two-level kernel's lanes b read Zech entries log b apart: multiples
    // of s = L/(q-1).  For s = 0 mod 4 those fall on few banks unless the
    // table carries one pad word per 32.
    uint32_t pad[kMaxG];
    for (uint32_t k = 0; k < j.g; ++k) pad[k] = (j.method == 2 && (j.L[k] / (j.q - 1)) % 4 == 0) ? 1u : 0u;
    auto words = [&](uint32_t k) -> uint64_t {
        uint64_t n = 0;
        if (kind[k] == kTabTripleSmem) n = 3ull * j.L[k] + 1;
        else if (kind[k] == kTabDoubleSmem) n = 2ull * j.L[k] + 1;
        else if (kind[k] == kTab17Smem) return (((j.L[k] + 2ull) & ~1ull) + 2 * ((j.L[k] + 32ull) / 32) + 7) / 8 * 8;
        else return 0;
        if (j.method == 2) n += kFan2Prefix;   // (method 2 never takes the 17-bit layout)
        if (pad[k]) n += 2 * ((n + 63) / 64);
        return ((n + 7) / 8) * 8;
    };
    // the two-level kernel for g = 4 and q <= 15 may stage a field's rows as
    // int16 (q digit bits, the flag in bit 15) when the u32 rows leave too
    // little room; such a field takes the doubled Zech layout and its orbit points
    uint32_t r16[kMaxG] = {0, 0, 0, 0};
    auto row_bytes = [&](uint32_t k) -> uint64_t {
        return j.method == 2 ? (r16[k] ? 2ull : 4ull) * (j.L[k] + kFan2ZeroRow + 1) : 4ull * j.words * (j.L[k] + 1);
    };
    auto fan_bytes = [&](void) -> uint64_t {
        if (j.method == 0) return 0;
        uint64_t b = 0;
        for (uint32_t k = 0; k < j.g; ++k) b += ((row_bytes(k) + 15) / 16) * 16 + ((j.q + 15) / 16) * 16;
        b += ((3ull * j.q * j.q + j.q + 15) / 16) * 16;
        if (j.method == 2 && j.g == 2 && j.coord2) b += ((4ull * j.L[1] + 15) / 16) * 16;
        if (j.method == 2) b += 16 + (uint64_t)kFan2WarpsHost * fan2_warp_bytes(j.q, false);   // smallest block
        return b;
    };
    // the class-sharing variant of the per-member kernel stages points per warp
    const uint64_t cls_bytes = (j.method == 0 && j.words == 1) ? 16ull + kClsMaxWarps * kClsWarpBytes : 0ull;
    auto bytes_for = [&](void) {
        uint64_t u16 = 0;
        for (uint32_t k = 0; k < j.g; ++k) u16 += words(k);
        return u16 * 2 + 4ull * j.g * ((j.q + 3) / 4) * 4 + fan_bytes() + cls_bytes;
    };
    // int16 rows, largest field first, while that makes room for 16 warps
    if (j.method == 2 && j.g == 4 && j.q <= 15) {
        const uint64_t extra = (uint64_t)(16 - kFan2WarpsHost) * fan2_warp_bytes(j.q, false);
        while (bytes_for() + extra > smem_limit) {
            int big = -1;
            for (uint32_t k = 0; k < j.g; ++k)
                if (!r16[k] && j.reps[k] && j.zech2[k] && (big < 0 || row_bytes(k) > row_bytes(big))) big = (int)k;
            if (big < 0) break;
            r16[big] = 1;
            kind[big] = kTabDoubleSmem;
        }
        // still short of 16 warps: int16-row fields give up the pad word when
        // the lanes' Zech reads (log b apart, word stride s / 2) already fall
        // on distinct banks (s / 2 not a multiple of 4)
        for (uint32_t k = 0; k < j.g && bytes_for() + extra > smem_limit; ++k) {
            const uint32_t s = j.L[k] / (j.q - 1);
            if (r16[k] && pad[k] && (s / 2) % 4 != 0) pad[k] = 0;
        }
    }
    // the two-level kernel reads its Zech tables only in the shared chain: give
    // up tripled tables, largest first, while that makes room for 16 warps
    if (j.method == 2) {
        const uint64_t extra = (uint64_t)(16 - kFan2WarpsHost) * fan2_warp_bytes(j.q, false);
        while (bytes_for() + extra > smem_limit) {
            int big = -1;
            for (uint32_t k = 0; k < j.g; ++k)
                if (kind[k] == kTabTripleSmem && j.zech2[k] && (big < 0 || words(k) > words(big))) big = (int)k;
            if (big < 0) break;
            kind[big] = kTabDoubleSmem;
        }
    }
    while (bytes_for() > smem_limit) {
        int big = -1;
        for (uint32_t k = 0; k < j.g; ++k)
            if (kind[k] != kTabDoubleGlobal && (big < 0 || words(k) > words(big))) big = (int)k;
        if (big < 0) break;
        kind[big] = (kind[big] == kTabTripleSmem && j.zech2[big]) ? kTabDoubleSmem
                    : (kind[big] != kTab17Smem && small17(big)) ? kTab17Smem
                                                                 : kTabDoubleGlobal;
    }
    if (bytes_for() > smem_limit) return false;
    if (j.method == 2)   // the two-level kernel reads every Zech table from shared memory
        for (uint32_t k = 0; k < j.g; ++k)
            if (kind[k] == kTabDoubleGlobal) return false;
    uint32_t off = 0;
    for (uint32_t k = 0; k < kMaxG; ++k) {
        j.tab_kind[k] = k < j.g ? kind[k] : kTabDoubleGlobal;
        j.tab_pad[k] = (k < j.g && kind[k] != kTabDoubleGlobal && kind[k] != kTab17Smem) ? pad[k] : 0u;
        j.row16[k] = k < j.g ? r16[k] : 0u;
        j.tab_off[k] = off;
        // 17-bit layout: L + 1 low halves (even count), then the high-bit plane
        j.tab_hi_off[k] = off + (k < j.g ? ((j.L[k] + 2u) & ~1u) : 0u);
        if (k < j.g) off += (uint32_t)words(k);
    }
    j.smem_u16 = off;
    uint32_t off32 = off / 2;
    for (uint32_t k = 0; k < kMaxG; ++k) {
        j.coef_off[k] = off32;
        if (k < j.g) off32 += ((j.q + 3) / 4) * 4;
    }
    uint32_t bytes = off32 * 4;   // multiple of 16
    for (uint32_t k = 0; k < kMaxG; ++k) {
        j.row_off[k] = bytes;
        j.zdig_off[k] = bytes;
        if (j.method != 0 && k < j.g) {
            bytes += (uint32_t)row_bytes(k);
            bytes = (bytes + 15) / 16 * 16;
            j.zdig_off[k] = bytes;
            bytes += ((j.q + 15) / 16) * 16;
        }
    }
    j.fq_off = bytes;
    if (j.method != 0) bytes += ((3 * j.q * j.q + j.q + 15) / 16) * 16;   // mul | sub | inv | add
    j.coord_off = 0;
    if (j.method == 2 && j.g == 2 && j.coord2) {   // coordinates of F_{q^2} (direct zero digits, g = 2)
        j.coord_off = bytes;
        bytes += ((4 * j.L[1] + 15) / 16) * 16;
    }
    j.warp_off = 0;
    j.warp_bytes = 0;
    j.dense_off = 0;
    if (j.method == 2) {
        bytes = (bytes + 15) / 16 * 16;
        // g <= 2: the CTA counts (a_1, a_2) in a dense box of shared counters
        // when that leaves room for 24 warps
        if (j.g <= 2) {
            const int32_t b1 = (int32_t)isqrt_u64(4ull * j.g * j.g * j.q);
            const int32_t b2 = j.g == 2 ? (int32_t)(2 * j.g * j.q) : 0;
            const uint32_t n = (uint32_t)(2 * b1 + 1) * (uint32_t)(2 * b2 + 1);
            const uint32_t dbytes = (4 * n + 15) / 16 * 16;
            if ((uint64_t)bytes + dbytes + 24ull * fan2_warp_bytes(j.q, true) + 16 <= smem_limit) {
                j.dense_off = bytes;
                j.dense_b1 = b1;
                j.dense_b2 = b2;
                j.dense_w2 = (uint32_t)(2 * b2 + 1);
                j.dense_n = n;
                bytes += dbytes;
            }
        }
        j.warp_off = bytes;
        j.warp_bytes = fan2_warp_bytes(j.q, j.dense_off != 0);
        bytes += kFan2WarpsHost * j.warp_bytes;
    }
    if (cls_bytes) {   // room for the largest block of the per-member kernels
        bytes = (bytes + 15) / 16 * 16;
        j.warp_off = bytes;
        j.warp_bytes = kClsWarpBytes;
        bytes += kClsMaxWarps * kClsWarpBytes;
    }
    j.smem_bytes = bytes;
    return true;
}

static uint32_t next_pow2(uint64_t v)
{
    uint64_t c = 1;
    while (c < v) c <<= 1;
    return (uint32_t)std::min<uint64_t>(c, 1ull << 31);
}

// number of (a_1..a_g) tuples allowed by the Hasse-Weil bound |a_k| <= 2g sqrt(q^k)
static uint64_t hasse_weil_box(uint32_t g, uint32_t q)
{
    double box = 1;
    double Q = 1;
    for (uint32_t k = 1; k <= g; ++k) {
        Q *= q;
        double b = std::floor(2.0 * g * std::sqrt(Q));
        box *= 2 * b + 1;
    }
    return box > 1e18 ? (uint64_t)1e18 : (uint64_t)box;
}

// Upper bound on the number of distinct keys (a_1..a_g) of square-free
// members for g <= 3: the L-polynomial of a curve of genus g determines them
// (Newton's identities) and has all roots of absolute value sqrt(q), so its
// real Weil polynomial h(x) = prod (x - r_i) is monic with integer
// coefficients (c_1, ..., c_g), an integer shift of the L-polynomial's, and
// all roots r_i real in [-m, m], m = 2 sqrt(q).  Counted by the admissible
// range of c_g for each (c_1, .., c_{g-1}), each range widened by one integer on
// both sides against rounding.  0 for g > 3 (not counted).
static uint64_t weil_poly_bound(uint32_t g, uint32_t q)
{
    const double m = 2.0 * std::sqrt((double)q);
    auto range = [](double lo, double hi) -> uint64_t {   // integers in [lo - 1, hi + 1]
        const double a = std::ceil(lo - 1.0), b = std::floor(hi + 1.0);
        return b >= a ? (uint64_t)(b - a) + 1 : 0;
    };
    if (g == 1) return 2 * (uint64_t)std::floor(m) + 3;
    const int64_t c1max = (int64_t)std::floor((double)g * m) + 1;
    uint64_t n = 0;
    if (g == 2) {
        // x^2 + c1 x + c2: real roots (c2 <= c1^2 / 4) in [-m, m] (h(+-m) >= 0)
        for (int64_t c1 = -c1max; c1 <= c1max; ++c1) {
            const double a = (double)c1;
            if (std::fabs(a) > 2 * m + 1) continue;
            n += range(m * std::fabs(a) - m * m, a * a / 4);
        }
        return n;
    }
    if (g == 3) {
        // x^3 + c1 x^2 + c2 x + c3 = f(x) + c3: both critical points in
        // [-m, m] and f(x_max) + c3 >= 0 >= f(x_min) + c3, f(-m) + c3 <= 0 <= f(m) + c3
        const int64_t c2lo = -(int64_t)std::ceil(3 * m * m) - 1, c2hi = (int64_t)std::ceil(3 * m * m) + 1;
        for (int64_t c1 = -c1max; c1 <= c1max; ++c1)
            for (int64_t c2 = c2lo; c2 <= c2hi; ++c2) {
                const double a = (double)c1, b = (double)c2;
                const double disc = a * a - 3 * b;
                if (disc < -1e-9) continue;
                const double sd = std::sqrt(std::max(disc, 0.0));
                const double x1 = (-a - sd) / 3, x2 = (-a + sd) / 3;
                if (x1 < -m - 1e-9 || x2 > m + 1e-9) continue;
                auto f = [&](double x) { return ((x + a) * x + b) * x; };
                n += range(std::max(-f(x1), -f(m)), std::min(-f(x2), -f(-m)));
            }
        return n;
    }
    return 0;
}

struct HostJob {
    hwc_job_t job;
    KJob kj;
    uint64_t fam_n;
    int warps = 0;   // tuned warps per CTA (two-level kernel)
    int block = 0;   // threads per CTA of the job's launch when it runs alone
};

void set_points(KJob &kj, uint32_t k, const Tables *t, bool orbits)
{
    const bool orb = orbits && k >= 2 && t->d_reps;
    kj.reps[k - 1] = orb ? t->d_reps : nullptr;
    kj.npts[k - 1] = orb ? t->n_reps : t->L;
    // the two-level kernel keeps the zeros of field m apart when some
    // S_k = ... + m (N_m - Z_m) needs them (k = 2m, 4m <= g): in bits s.. of
    // its accumulators, 2^s above 2 (points) + (zeros <= d)
    kj.zshift[k - 1] = 0;
    if (orbits && 2 * k <= kj.g) {
        uint32_t s = 0;
        while ((1u << s) <= 2 * kj.npts[k - 1] + kj.d) ++s;
        kj.zshift[k - 1] = s;
    }
}

// the pattern table of the reduced family (HWC_FAM_REDUCED, hwc.h): starts,
// patterns, gcd(q-1, i-j), mult, and the digits w^t of the smallest digit w
// generating F_q^x (read off the logs of the digits in F_q)
static int fill_reduced(KJob &kj, const Tables *t1)
{
    const uint32_t q = kj.q, d = kj.d;
    std::vector<uint32_t> lg(q);
    HWC_CUDA_TRY(cudaMemcpy(lg.data(), t1->d_coef_log, q * sizeof(uint32_t), cudaMemcpyDeviceToHost));
    const uint32_t L = q - 1;
    uint32_t w = 1;
    for (uint32_t c = 2; c < q; ++c)
        if (lg[c] < L && std::gcd(lg[c], L) == 1) { w = c; break; }
    std::vector<uint32_t> digit_of_log(L, 0);
    for (uint32_t c = 1; c < q; ++c) digit_of_log[lg[c] % L] = c;
    for (uint32_t t = 0; t < 2 * (uint32_t)kMaxG; ++t) kj.red_w[t] = digit_of_log[(uint64_t)t * lg[w] % L];
    uint32_t n = 0;
    uint64_t start = 0;
    const uint64_t m1 = (uint64_t)q * (q - 1) / 2;
    auto add = [&](uint32_t i, uint32_t j, uint32_t gg, uint64_t size, uint64_t mult) {
        kj.red_start[n] = start;
        kj.red_i[n] = (uint8_t)i;
        kj.red_j[n] = (uint8_t)j;
        kj.red_gcd[n] = (uint8_t)gg;
        kj.red_mult[n] = mult;
        start += size;
        ++n;
    };
    add(0xFF, 0, 1, q - 1, m1);   // A: c_d X^d + 1
    add(0xFE, 0, 1, q - 1, m1);   // B: c_d X^d + X
    for (uint32_t i = 1; i + 2 <= d; ++i)
        for (uint32_t j = 0; j < i; ++j) {
            const uint32_t gg = std::gcd(q - 1, i - j);
            uint64_t qj = 1;
            for (uint32_t e = 0; e < j; ++e) qj *= q;
            add(i, j, gg, (uint64_t)(q - 1) * gg * qj, (uint64_t)q * (q - 1) * (q - 1) / (2 * gg));
        }
    kj.red_n = n;
    kj.red_start[n] = start;
    return HWC_OK;
}

int fill_kjob(const hwc_job_t &jb, KJob &kj, uint64_t *fam_n, uint32_t flags, const TuneChoice *tc)
{
    int rc = validate_job(jb, fam_n);
    if (rc) return rc;
    std::memset(&kj, 0, sizeof kj);
    uint32_t p, e;
    prime_power(jb.q, &p, &e);
    kj.g = jb.g;
    kj.q = jb.q;
    kj.d = jb.family.degree;
    kj.kind = jb.family.kind;
    kj.p = p;
    kj.seed = jb.family.seed;
    kj.first = jb.first;
    kj.count = jb.count;
    upow(jb.q, kj.d - 1, &kj.fam_mz);
    kj.qd = kj.fam_mz * jb.q;
    kj.n_tiles = (jb.count + kTileMembers - 1) / kTileMembers;
    if ((flags & HWC_FLAG_LAMBDA) && (flags & HWC_FLAG_ALL_POINTS))
        return set_error(HWC_ERR_ARG, "HWC_FLAG_LAMBDA needs the Frobenius-orbit points (not HWC_FLAG_ALL_POINTS)");
    if (flags & HWC_FLAG_LAMBDA) {
        // key: a_k + B_k in just enough bits per field, then n_1..n_g and the split bit
        kj.lam_mode = 1;
        uint32_t off = 0;
        double Qk = 1;
        for (uint32_t k = 0; k < jb.g; ++k) {
            Qk *= jb.q;
            const int32_t B = (int32_t)std::floor(2.0 * jb.g * std::sqrt(Qk));
            uint32_t w = 0;
            while ((1ull << w) <= 2ull * (uint64_t)B) ++w;
            kj.key_bias[k] = B;
            kj.key_shift[k] = off;
            off += w;
        }
        kj.lam_shift = off;
        if (off + 4 * jb.g + 1 > 63) return set_error(HWC_ERR_TOO_LARGE, "lambda key needs %u bits", off + 4 * jb.g + 1);
    }
    // enumerated families with q <= 63: groups of q members share all but c_0
    const bool window = jb.family.kind == HWC_FAM_MONIC_NOSUB_SAMPLED_WINDOW;
    const bool fan = !(flags & (HWC_FLAG_HORNER | HWC_FLAG_LAMBDA)) && jb.family.kind != HWC_FAM_MONIC_NOSUB_SAMPLED &&
                     !window &&
                     jb.family.kind != HWC_FAM_REDUCED && jb.q <= 63 &&
                     !(tc && tc->method == 0);
    const bool no_triple = tc && tc->no_triple;
    // (method chosen below: two-level fan-out for q <= 31, one-level up to 63,
    // per-member Horner otherwise or when a layout does not fit)
    for (uint32_t k = 1; k <= jb.g; ++k) {
        const Tables *t = nullptr;
        rc = tables_cached(jb.q, k, &t);
        if (rc) return rc;
        kj.Q[k - 1] = t->Q;
        kj.L[k - 1] = t->L;
        kj.barrett[k - 1] = (uint32_t)((1ull << 32) / t->L);
        kj.zech2[k - 1] = t->d_zech2;
        kj.zech3[k - 1] = t->d_zech3;
        kj.zech2w[k - 1] = t->d_zech2w;
        kj.coef_log[k - 1] = t->d_coef_log;
        kj.z17lo[k - 1] = t->d_z17lo;
        kj.z17hi[k - 1] = t->d_z17hi;
        set_points(kj, k, t, !(flags & HWC_FLAG_ALL_POINTS));
        kj.rows[k - 1] = jb.q <= 31 ? (const void *)t->d_rows32 : (const void *)t->d_rows64;
        if (k == 1) {
            kj.fq_mul = t->d_fq_mul;
            kj.fq_sub = t->d_fq_sub;
            kj.fq_inv = t->d_fq_inv;
        }
        kj.zdig[k - 1] = t->d_zdig;
        if (k == 2) kj.coord2 = t->d_coord2;
        if (k == 1 && jb.family.kind == HWC_FAM_REDUCED && (rc = fill_reduced(kj, t))) return rc;
        // ceil(2^32 / s) recovers l / s exactly for multiples l of s = L/(q-1) < 2^32;
        // s = 1 (k = 1) is encoded as 0
        const uint32_t sdiv = t->L / (jb.q - 1);
        kj.zdiv[k - 1] = sdiv == 1 ? 0u : (uint32_t)(((1ull << 32) + sdiv - 1) / sdiv);
    }
    const uint32_t limit = device_smem_optin() - 4096;   // static smem of the kernels
    // a sampled family with q <= 31 drawn densely (at least one sample per 32
    // members): the two-level kernel counts every member of the family once,
    // with its multiplicity among the samples as weight (the weights take 4
    // bytes per member, at most 16 GB; fewer than 2^27 samples keep the sums
    // of 32 weights below 2^32)
    const bool weighted = jb.family.kind == HWC_FAM_MONIC_NOSUB_SAMPLED && jb.q <= 31 &&
                          !(flags & (HWC_FLAG_HORNER | HWC_FLAG_FAN1 | HWC_FLAG_LAMBDA | kFlagNoWeights)) &&
                          !(tc && tc->method >= 0 && tc->method != 2) && jb.count >= kj.fam_mz / 32 &&
                          jb.count < (1ull << 27) && kj.fam_mz <= (1ull << 32);
    if (window) {   // the draws of the whole sample in a window of members: the weighted kernel only
        const uint64_t qq = (uint64_t)jb.q * jb.q;
        const uint64_t sc = jb.family.sample_count;
        if (jb.q > 31 || (flags & (HWC_FLAG_HORNER | HWC_FLAG_FAN1 | HWC_FLAG_LAMBDA | kFlagNoWeights)) ||
            (tc && tc->method >= 0 && tc->method != 2) || sc < kj.fam_mz / 32 || sc >= (1ull << 27) ||
            kj.fam_mz > (1ull << 32))
            return set_error(HWC_ERR_ARG, "a windowed sampled family runs only on the whole-family kernel "
                                          "(q <= 31, at least one draw per 32 members, fewer than 2^27 draws)");
        kj.method = 2;
        kj.words = 2;
        kj.s_first = 0;
        kj.s_count = sc;
        kj.w_first = jb.first;
        kj.w_n = jb.count;
        kj.first_group = jb.first / qq;
        kj.n_tiles = jb.count ? (jb.first + jb.count - 1) / qq - kj.first_group + 1 : 0;
        if (layout_job_smem(kj, limit, no_triple)) return HWC_OK;
        return set_error(HWC_ERR_ARG, "the tables of a windowed sampled family do not fit in shared memory");
    }
    if (weighted) {
        const uint64_t qq = (uint64_t)jb.q * jb.q;
        kj.method = 2;
        kj.words = 2;   // the weighted instantiation of the two-level kernel
        kj.s_first = jb.first;
        kj.s_count = jb.count;
        kj.first = 0;
        kj.count = kj.fam_mz;
        kj.w_first = 0;
        kj.w_n = kj.fam_mz;
        kj.first_group = 0;
        kj.n_tiles = kj.fam_mz / qq;
        if (layout_job_smem(kj, limit, no_triple)) return HWC_OK;
        kj.first = jb.first;   // tables do not fit: per-member Horner over the samples
        kj.count = jb.count;
        kj.s_first = kj.s_count = 0;
        kj.w_first = kj.w_n = 0;
        kj.first_group = 0;
        kj.method = 0;
        kj.words = 0;
        kj.n_tiles = (jb.count + kTileMembers - 1) / kTileMembers;
    }
    if (fan && jb.q <= 31 && !(flags & HWC_FLAG_FAN1) && !(tc && tc->method == 1)) {
        // two-level fan-out: groups of q^2 members
        kj.method = 2;
        kj.words = 1;
        kj.first_group = jb.first / ((uint64_t)jb.q * jb.q);
        kj.n_tiles = jb.count ? (jb.first + jb.count - 1) / ((uint64_t)jb.q * jb.q) - kj.first_group + 1 : 0;
        if (layout_job_smem(kj, limit, no_triple)) return HWC_OK;
    }
    if (fan) {
        kj.method = 1;
        kj.words = jb.q <= 31 ? 1 : 2;
        kj.first_group = jb.first / jb.q;
        kj.n_tiles = jb.count ? (jb.first + jb.count - 1) / jb.q - kj.first_group + 1 : 0;
        if (layout_job_smem(kj, limit, no_triple)) return HWC_OK;
        kj.method = 0;   // rows do not fit: per-member Horner
        kj.words = 0;
        kj.first_group = 0;
        kj.n_tiles = (jb.count + kTileMembers - 1) / kTileMembers;
    }
    // a sparse sample with many draws per class of high digits (c_2..c_{d-2}):
    // the class-sharing variant of the per-member kernel (doubled tables)
    if (kj.method == 0 && jb.family.kind == HWC_FAM_MONIC_NOSUB_SAMPLED && kj.d >= 3 && kj.d <= 6 &&
        !(flags & (HWC_FLAG_HORNER | HWC_FLAG_LAMBDA | kFlagNoWeights | kFlagNoClass)) &&
        jb.count < (1ull << 27)) {
        uint64_t ncls = 1;
        if (upow(jb.q, kj.d - 3, &ncls) && ncls < (1ull << 31) && jb.count >= kClsMinPerClass * ncls) {
            kj.words = 1;
            kj.cls_n = (uint32_t)ncls;
            kj.n_tiles = (jb.count + 31) / 32 + ncls;
            if (layout_job_smem(kj, limit, true)) return HWC_OK;
            kj.words = 0;
            kj.cls_n = 0;
            kj.n_tiles = (jb.count + kTileMembers - 1) / kTileMembers;
        }
    }
    layout_job_smem(kj, limit, no_triple);
    return HWC_OK;
}

uint32_t hash_capacity(uint32_t g, uint32_t q, uint64_t count, uint32_t scale)
{
    uint64_t bound = std::min<uint64_t>(count, hasse_weil_box(g, q));
    const uint64_t weil = weil_poly_bound(g, q);
    if (weil) bound = std::min(bound, weil);
    uint32_t cap = next_pow2(std::max<uint64_t>(256, 2 * bound * scale));
    return std::min<uint32_t>(cap, 1u << 28);
}

}  // namespace hwc

using namespace hwc;

// ---------------------------------------------------------------------
// histograms

// entries keyed by (pattern code, tuple); without patterns the code is 0
using HistMap = std::map<std::pair<uint64_t, std::vector<int32_t>>, uint64_t>;

static hwc_hist *hist_from_map(uint32_t g, const HistMap &m, uint64_t n_total, bool has_lam)
{
    hwc_hist *h = new hwc_hist();
    h->g = g;
    h->n_total = n_total;
    h->has_lam = has_lam;
    h->counts.reserve(m.size() * g);
    h->mult.reserve(m.size());
    for (auto &kv : m) {
        h->counts.insert(h->counts.end(), kv.first.second.begin(), kv.first.second.end());
        if (has_lam) h->lam.push_back(kv.first.first);
        h->mult.push_back(kv.second);
        h->n_sqf += kv.second;
    }
    return h;
}

// the full pattern code of eq. 1.2 from a lambda-mode key: n_1..n_g, the
// degree left over (one factor, or two of degree g+1 with the split bit) and
// the extra part 1 of odd degree
static uint64_t lambda_code(const KJob &kj, uint64_t key)
{
    const uint32_t g = kj.g, d = kj.d;
    uint32_t n[2 * kMaxG + 3] = {};
    uint32_t used = 0;
    for (uint32_t m = 1; m <= g; ++m) {
        n[m] = (uint32_t)(key >> (kj.lam_shift + 4 * (m - 1))) & 0xFu;
        used += m * n[m];
    }
    const bool split = (key >> (kj.lam_shift + 4 * g)) & 1u;
    if (used < d) {
        if (split) n[g + 1] += 2;
        else n[d - used] += 1;
    }
    if (d == 2 * g + 1) n[1] += 1;
    uint64_t code = 0;
    for (uint32_t m = 1; m <= 2 * g + 2; ++m) code += (uint64_t)n[m] << (4 * (m - 1));
    return code;
}

hwc_hist *hwc::hist_from_keys(const KJob &kj, const unsigned long long *keys,
                              const unsigned long long *cnt, uint64_t n, uint64_t n_total)
{
    if (kj.lam_mode) {   // (a_1..a_g, lambda) keys: decode, then sort by (pattern, tuple)
        HistMap m;
        for (uint64_t i = 0; i < n; ++i) {
            std::vector<int32_t> t(kj.g);
            for (uint32_t k = 0; k < kj.g; ++k) {
                const uint32_t w = (k + 1 < kj.g ? kj.key_shift[k + 1] : kj.lam_shift) - kj.key_shift[k];
                const int a = (int)((keys[i] >> kj.key_shift[k]) & ((1ull << w) - 1)) - kj.key_bias[k];
                t[k] = (int32_t)kj.Q[k] + 1 - a;   // #C = Q + 1 - a (eq. 1.1)
            }
            m[{lambda_code(kj, keys[i]), t}] += cnt[i];
        }
        return hist_from_map(kj.g, m, n_total, true);
    }
    // #C_k = Q_k + 1 - a_k (eq. 1.1) and key slot k holds a_k + 32768, so the
    // tuples in lexicographic order of (#C_1, ..., #C_g) are the keys in
    // ascending order of sum_k (0xFFFF - slot_k) 2^(16 (g-1-k)): one sort of
    // 64-bit words
    const uint32_t g = kj.g;
    std::vector<std::pair<uint64_t, uint64_t>> ord(n);
    for (uint64_t i = 0; i < n; ++i) {
        uint64_t t = 0;
        for (uint32_t k = 0; k < g; ++k) t = (t << 16) | (0xFFFFu - ((keys[i] >> (16 * k)) & 0xFFFFu));
        ord[i] = {t, cnt[i]};
    }
    std::sort(ord.begin(), ord.end());
    hwc_hist *h = new hwc_hist();
    h->g = g;
    h->n_total = n_total;
    h->counts.resize(n * g);
    h->mult.resize(n);
    for (uint64_t i = 0; i < n; ++i) {
        const uint64_t t = ord[i].first;
        for (uint32_t k = 0; k < g; ++k) {
            const int a = (int)(0xFFFFu - ((t >> (16 * (g - 1 - k))) & 0xFFFFu)) - 32768;
            h->counts[i * g + k] = (int32_t)kj.Q[k] + 1 - a;
        }
        h->mult[i] = ord[i].second;
        h->n_sqf += ord[i].second;
    }
    return h;
}

// ---------------------------------------------------------------------
// batches

// Jobs of one degree share a persistent launch (the kernel is specialised on
// the degree); a batch holds one group per distinct degree.
struct BatchGroup {
    int D = 0;
    uint32_t method = 0, words = 0;
    int block = 0;                   // the jobs' own block size (one launch per block size)
    int warps = 0;                   // tuned warps per CTA (two-level kernel)
    uint64_t warps_tiles = 0;        // groups of the job that set `warps`
    uint32_t first = 0, n = 0;       // jobs[first .. first+n) (sorted by degree)
    uint32_t start_off = 0;          // offset of this group's item table
    uint64_t n_items = 0;
    uint32_t max_smem = 0;
    LaunchShape shape;
};

struct hwc_batch {
    std::vector<HostJob> jobs;       // sorted by degree
    std::vector<size_t> pos;         // caller's index -> position in jobs
    std::vector<BatchGroup> groups;
    KJob *h_jobs = nullptr;          // pinned copy of the descriptors
    uint64_t *h_item_start = nullptr;
    size_t n_starts = 0;
    KJob *d_jobs = nullptr;
    uint64_t *d_item_start = nullptr;
    unsigned long long *d_counters = nullptr;
    std::vector<void *> allocs;
    uint32_t flags = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    cudaEvent_t done = nullptr;
    cudaEvent_t t0 = nullptr, t1 = nullptr;   // HWC_FLAG_TIMING
    bool launched = false;
    uint64_t d2h_last = 0;
    int device = 0;
    uint32_t launches_per_run = 0;
    uint32_t weight_launches = 0;    // sampled jobs whose multiplicities are scattered each run
    // persistent batches with several launch groups: the groups after the
    // first run on side streams (forked from and joined to the launch
    // stream), so the tail of one launch overlaps the others
    std::vector<cudaStream_t> side;
    std::vector<cudaEvent_t> side_done;
    cudaEvent_t fork = nullptr;
};

static void batch_release(hwc_batch *b)
{
    if (!b) return;
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->done) cudaEventDestroy(b->done);
    if (b->t0) cudaEventDestroy(b->t0);
    if (b->t1) cudaEventDestroy(b->t1);
    if (b->h_jobs) cudaFreeHost(b->h_jobs);
    if (b->h_item_start) cudaFreeHost(b->h_item_start);
    for (cudaStream_t st : b->side) cudaStreamDestroy(st);
    for (cudaEvent_t ev : b->side_done) cudaEventDestroy(ev);
    if (b->fork) cudaEventDestroy(b->fork);
    for (void *p : b->allocs) cudaFree(p);
    delete b;
}

template <class T>
static int dalloc(hwc_batch *b, T **p, uint64_t n)
{
    void *v = nullptr;
    if (cudaMalloc(&v, std::max<uint64_t>(n, 1) * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        return set_error(HWC_ERR_NOMEM, "cudaMalloc of %llu bytes failed",
                         (unsigned long long)(n * sizeof(T)));
    }
    b->allocs.push_back(v);
    *p = (T *)v;
    return HWC_OK;
}

static int batch_enqueue(hwc_batch *b, cudaStream_t s, bool capturing)
{
    const uint32_t nj = (uint32_t)b->jobs.size();
    // the step's inputs: job descriptors and the work-item tables, from pinned memory
    HWC_CUDA_TRY(cudaMemcpyAsync(b->d_jobs, b->h_jobs, nj * sizeof(KJob), cudaMemcpyHostToDevice, s));
    HWC_CUDA_TRY(cudaMemcpyAsync(b->d_item_start, b->h_item_start, b->n_starts * sizeof(uint64_t),
                                 cudaMemcpyHostToDevice, s));
    int rc = launch_clear(b->d_jobs, nj, b->d_counters, (uint32_t)b->groups.size(), s);
    if (rc) return rc;
    for (const HostJob &hj : b->jobs)   // multiplicities of the samples counted over whole families
        if ((rc = launch_sample_weights(hj.kj, s)) || (rc = launch_class_sort(hj.kj, s))) return rc;
    // inside a graph capture an event record must be an external node to time anything
    if (b->t0) HWC_CUDA_TRY(capturing ? cudaEventRecordWithFlags(b->t0, s, cudaEventRecordExternal)
                                      : cudaEventRecord(b->t0, s));
    const bool fork = !b->side.empty();
    if (fork) HWC_CUDA_TRY(cudaEventRecord(b->fork, s));
    for (size_t g = 0; g < b->groups.size(); ++g) {
        const BatchGroup &G = b->groups[g];
        cudaStream_t gs = s;
        if (fork && g > 0) {
            gs = b->side[g - 1];
            HWC_CUDA_TRY(cudaStreamWaitEvent(gs, b->fork, 0));
        }
        rc = launch_persistent(G.D, G.method, G.words, b->d_jobs + G.first, b->d_item_start + G.start_off, G.n,
                               G.n_items, b->d_counters + g, G.max_smem, G.shape, gs);
        if (rc) return rc;
        if (fork && g > 0) HWC_CUDA_TRY(cudaEventRecord(b->side_done[g - 1], gs));
    }
    if (fork)
        for (cudaEvent_t ev : b->side_done) HWC_CUDA_TRY(cudaStreamWaitEvent(s, ev, 0));
    if (b->t1) HWC_CUDA_TRY(capturing ? cudaEventRecordWithFlags(b->t1, s, cudaEventRecordExternal)
                                      : cudaEventRecord(b->t1, s));
    return launch_compact(b->d_jobs, nj, s);
}

// threads per CTA that maximise resident warps per SM for this degree and smem
int hwc::choose_shape(int D, uint32_t method, uint32_t words, uint32_t smem, bool persistent, LaunchShape *out)
{
    const int sms = device_sm_count();
    int best_block = 256, best_warps = -1, best_ctas = 1;
    // per-member kernel: 256 threads unless only a larger block keeps more
    // warps resident (one CTA per SM for the 17-bit tables)
    const int blocks[4] = {method == 2 ? kFan2WarpsHost * 32 : 256, 128, 512, 768};
    for (int bi = 0; bi < (method == 0 ? 4 : 1); ++bi) {
        const int block = blocks[bi];
        int ctas = 0;
        int rc = max_ctas_per_sm(D, method, words, block, smem, persistent, &ctas);
        if (rc) return rc;
        const int warps = ctas * block / 32;
        if (warps > best_warps) {
            best_warps = warps;
            best_block = block;
            best_ctas = ctas;
        }
    }
    if (best_warps <= 0) return set_error(HWC_ERR_TOO_LARGE, "no CTA fits %u bytes of shared memory", smem);
    out->block = best_block;
    out->grid = sms * best_ctas;
    out->item_tiles = (best_block / 32) * (method == 0 ? 2 : 1);
    return HWC_OK;
}

int hwc::choose_shape_fan2(int D, const Fan2Need *needs, size_t n, LaunchShape *out, uint32_t *smem, int warps)
{
    const int sms = device_sm_count();
    const uint32_t limit = device_smem_optin() - 4096;
    int best_warps = -1;
    for (int block : {768, 512, 384, 256, 128}) {
        if (warps > 0 && block != 32 * warps) continue;   // the tuned block
        const uint32_t W = (uint32_t)block / 32;
        uint32_t need = 0;
        for (size_t i = 0; i < n; ++i) need = std::max(need, needs[i].warp_off + W * needs[i].warp_bytes);
        if (need > limit) continue;
        int ctas = 0;
        int rc = max_ctas_per_sm(D, 2, 1, block, need, true, &ctas);
        if (rc) return rc;
        if (ctas * (int)W > best_warps) {
            best_warps = ctas * (int)W;
            out->block = block;
            out->grid = sms * ctas;
            out->item_tiles = (int)W;
            *smem = need;
        }
    }
    if (best_warps <= 0) {
        if (warps > 0) return choose_shape_fan2(D, needs, n, out, smem, 0);   // the tuned block no longer fits
        return set_error(HWC_ERR_TOO_LARGE, "no CTA of the two-level kernel fits");
    }
    return HWC_OK;
}

static int batch_create_impl(const hwc_job_t *jobs, size_t n, uint32_t flags, uint32_t cap_scale,
                             hwc_batch **out, const TuneChoice *given = nullptr)
{
    *out = nullptr;
    if (!jobs || n == 0) return set_error(HWC_ERR_ARG, "no jobs");
    for (size_t i = 0; i < n; ++i) {   // argument errors before any CUDA call
        uint64_t fam_n = 0;
        int vrc = validate_job(jobs[i], &fam_n);
        if (vrc) return vrc;
    }
    int rc = prepare_count_kernels();
    if (rc) return rc;
    hwc_batch *b = new hwc_batch();
    b->flags = flags;
    cudaGetDevice(&b->device);
    // descriptors in the caller's order, then ordered by kernel (degree, method,
    // row width) so that jobs of one kernel share a persistent launch
    std::vector<HostJob> filled(n);
    for (size_t i = 0; i < n; ++i) {
        filled[i].job = jobs[i];
        TuneChoice tc;
        if (given) {
            tc = *given;
        } else if (!(flags & HWC_FLAG_NO_TUNE)) {
            rc = tune_choice(jobs[i], flags, &tc);
            if (rc) { batch_release(b); return rc; }
        }
        rc = fill_kjob(jobs[i], filled[i].kj, &filled[i].fam_n, flags, &tc);
        if (rc) { batch_release(b); return rc; }
        filled[i].warps = tc.warps;
        // the block size this job would launch with alone: jobs that prefer
        // different blocks get launches of their own (run side by side)
        const KJob &k = filled[i].kj;
        LaunchShape sh;
        uint32_t smem = k.smem_bytes;
        if (k.method == 2) {
            const Fan2Need need{k.warp_off, k.warp_bytes};
            rc = choose_shape_fan2((int)k.d, &need, 1, &sh, &smem, tc.warps);
        } else {
            rc = choose_shape((int)k.d, k.method, k.words, k.smem_bytes, true, &sh);
        }
        if (rc) { batch_release(b); return rc; }
        filled[i].block = sh.block;
    }
    std::vector<size_t> order(n);
    std::iota(order.begin(), order.end(), 0);
    auto gkey = [&](size_t x) {
        const KJob &k = filled[x].kj;
        return std::make_tuple(k.d, k.method, k.words, filled[x].block);
    };
    // within a launch the queue hands out the jobs' work items in this order:
    // the costliest items first (point evaluations per tile), so that the
    // cheap ones fill the tail of the launch
    auto item_cost = [&](size_t x) {
        const KJob &k = filled[x].kj;
        double pts = 0;
        for (uint32_t i = 0; i < k.g; ++i) pts += k.npts[i] + 1.0;
        const double members = k.method == 2 ? (double)k.q * k.q : k.method == 1 ? (double)k.q : (double)kTileMembers;
        return members * pts;
    };
    std::stable_sort(order.begin(), order.end(), [&](size_t x, size_t y) {
        if (gkey(x) != gkey(y)) return gkey(x) < gkey(y);
        return item_cost(x) > item_cost(y);
    });
    b->pos.resize(n);
    b->jobs.resize(n);
    for (size_t r = 0; r < n; ++r) {
        const size_t i = order[r];
        b->pos[i] = r;
        HostJob &hj = b->jobs[r];
        hj = filled[i];
        KJob &kj = hj.kj;
        const uint32_t cap = hash_capacity(kj.g, kj.q, jobs[i].count, cap_scale);
        kj.hmask = cap - 1;
        if ((rc = dalloc(b, &kj.hkeys, cap)) || (rc = dalloc(b, &kj.hcounts, cap)) ||
            (rc = dalloc(b, &kj.stats, 4)) || (rc = dalloc(b, &kj.out_keys, cap)) ||
            (rc = dalloc(b, &kj.out_counts, cap)) || (rc = dalloc(b, &kj.n_out, 1)) ||
            (needs_weights(kj) && (rc = dalloc(b, &kj.mweight, kj.w_n))) ||
            (kj.cls_n && ((rc = dalloc(b, &kj.cls_cnt, kj.cls_n)) || (rc = dalloc(b, &kj.cls_tiles, kj.n_tiles)) ||
                          (rc = dalloc(b, &kj.cls_sorted, kj.count))))) {
            batch_release(b);
            return rc;
        }
        if (needs_weights(kj)) ++b->weight_launches;
        // plain runs: every job is a group of its own (one launch per job)
        if (b->groups.empty() || (flags & HWC_FLAG_PLAIN) || b->groups.back().D != (int)kj.d ||
            b->groups.back().method != kj.method || b->groups.back().words != kj.words ||
            b->groups.back().block != hj.block) {
            BatchGroup G;
            G.D = (int)kj.d;
            G.method = kj.method;
            G.words = kj.words;
            G.block = hj.block;
            G.first = (uint32_t)r;
            b->groups.push_back(G);
        }
        BatchGroup &G = b->groups.back();
        G.n++;
        G.max_smem = std::max(G.max_smem, kj.smem_bytes);
        // warps per CTA are a property of the launch: the tuned value of the
        // group's largest job
        if (kj.method == 2 && kj.n_tiles >= G.warps_tiles) {
            G.warps_tiles = kj.n_tiles;
            G.warps = hj.warps;
        }
    }
    const bool persistent = !(flags & HWC_FLAG_PLAIN);
    std::vector<uint64_t> starts;
    for (BatchGroup &G : b->groups) {
        if (G.method == 2) {
            std::vector<Fan2Need> needs;
            uint32_t max_qq = 0;
            for (uint32_t r = G.first; r < G.first + G.n; ++r) {
                needs.push_back({b->jobs[r].kj.warp_off, b->jobs[r].kj.warp_bytes});
                max_qq = std::max(max_qq, b->jobs[r].kj.q * b->jobs[r].kj.q);
            }
            if ((rc = choose_shape_fan2(G.D, needs.data(), needs.size(), &G.shape, &G.max_smem, G.warps))) {
                batch_release(b);
                return rc;
            }
            // one key slot per resident warp of the launch
            unsigned long long *wk = nullptr;
            if ((rc = dalloc(b, &wk, (uint64_t)G.shape.grid * (G.shape.block / 32) * max_qq))) {
                batch_release(b);
                return rc;
            }
            for (uint32_t r = G.first; r < G.first + G.n; ++r) {
                b->jobs[r].kj.wkeys = wk;
                b->jobs[r].kj.wkeys_stride = max_qq;
            }
        } else if ((rc = choose_shape(G.D, G.method, G.words, G.max_smem, persistent, &G.shape))) {
            batch_release(b);
            return rc;
        }
        // work items: each job is cut into items of item_tiles tiles, in job order
        G.start_off = (uint32_t)starts.size();
        uint64_t acc = 0;
        for (uint32_t r = G.first; r < G.first + G.n; ++r) {
            starts.push_back(acc);
            acc += (b->jobs[r].kj.n_tiles + G.shape.item_tiles - 1) / G.shape.item_tiles;
        }
        starts.push_back(acc);
        G.n_items = acc;
    }
    b->n_starts = starts.size();
    if ((rc = dalloc(b, &b->d_jobs, n)) || (rc = dalloc(b, &b->d_item_start, b->n_starts)) ||
        (rc = dalloc(b, &b->d_counters, b->groups.size()))) {
        batch_release(b);
        return rc;
    }
    if (cudaMallocHost(&b->h_jobs, n * sizeof(KJob)) != cudaSuccess ||
        cudaMallocHost(&b->h_item_start, b->n_starts * sizeof(uint64_t)) != cudaSuccess) {
        cudaGetLastError();
        batch_release(b);
        return set_error(HWC_ERR_NOMEM, "pinned host allocation failed");
    }
    for (size_t r = 0; r < n; ++r) b->h_jobs[r] = b->jobs[r].kj;
    std::copy(starts.begin(), starts.end(), b->h_item_start);
    if (flags & HWC_FLAG_TIMING) {
        if (cudaEventCreate(&b->t0) != cudaSuccess || cudaEventCreate(&b->t1) != cudaSuccess) {
            batch_release(b);
            return set_error(HWC_ERR_CUDA, "cudaEventCreate failed");
        }
    }
    b->launches_per_run = 2 + (uint32_t)b->groups.size() + b->weight_launches;
    if (!(flags & HWC_FLAG_PLAIN) && b->groups.size() > 1) {   // plain runs stay one launch after another
        bool ok = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) == cudaSuccess;
        for (size_t g = 1; ok && g < b->groups.size(); ++g) {
            cudaStream_t st = nullptr;
            cudaEvent_t ev = nullptr;
            ok = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess;
            if (ok) b->side.push_back(st);
            ok = ok && cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess;
            if (ok) b->side_done.push_back(ev);
        }
        if (!ok) {
            batch_release(b);
            return set_error(HWC_ERR_CUDA, "side streams of the batch could not be created");
        }
    }
    if (cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming) != cudaSuccess) {
        batch_release(b);
        return set_error(HWC_ERR_CUDA, "cudaEventCreate failed");
    }
    if (flags & HWC_FLAG_GRAPH) {
        cudaStream_t cs;
        if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
            batch_release(b);
            return set_error(HWC_ERR_CUDA, "cudaStreamCreate failed");
        }
        cudaError_t ce = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (ce == cudaSuccess) {
            rc = batch_enqueue(b, cs, true);
            cudaError_t ce2 = cudaStreamEndCapture(cs, &b->graph);
            if (rc == HWC_OK && ce2 == cudaSuccess)
                ce = cudaGraphInstantiate(&b->gexec, b->graph, 0);
            else if (ce2 != cudaSuccess)
                ce = ce2;
        }
        cudaStreamDestroy(cs);
        if (rc != HWC_OK || ce != cudaSuccess) {
            batch_release(b);
            return rc ? rc : set_error(HWC_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(ce));
        }
    }
    *out = b;
    return HWC_OK;
}

static int batch_result_impl(hwc_batch *b, size_t i, hwc_hist **out)
{
    *out = nullptr;
    if (!b->launched) return set_error(HWC_ERR_STATE, "batch was not launched");
    if (i >= b->jobs.size()) return set_error(HWC_ERR_ARG, "job %zu out of range", i);
    HWC_CUDA_TRY(cudaEventSynchronize(b->done));
    const KJob &kj = b->jobs[b->pos[i]].kj;
    unsigned long long st[3] = {}, n_out = 0;
    HWC_CUDA_TRY(cudaMemcpy(st, kj.stats, sizeof st, cudaMemcpyDeviceToHost));
    HWC_CUDA_TRY(cudaMemcpy(&n_out, kj.n_out, sizeof n_out, cudaMemcpyDeviceToHost));
    if (st[2]) return set_error(HWC_ERR_TOO_LARGE, "histogram hash of job %zu overflowed", i);
    std::vector<unsigned long long> keys(n_out), cnt(n_out);
    if (n_out) {
        HWC_CUDA_TRY(cudaMemcpy(keys.data(), kj.out_keys, n_out * 8, cudaMemcpyDeviceToHost));
        HWC_CUDA_TRY(cudaMemcpy(cnt.data(), kj.out_counts, n_out * 8, cudaMemcpyDeviceToHost));
    }
    if (i == 0) b->d2h_last = 0;
    b->d2h_last += sizeof st + sizeof n_out + 16 * n_out;
    hwc_hist *h = hist_from_keys(kj, keys.data(), cnt.data(), n_out, st[0]);
    if (h->n_sqf != st[1]) {
        uint64_t got = h->n_sqf;
        delete h;
        return set_error(HWC_ERR_CUDA, "histogram total %llu != square-free count %llu",
                         (unsigned long long)got, (unsigned long long)st[1]);
    }
    *out = h;
    return HWC_OK;
}

int hwc::batch_create_with(const hwc_job_t *jobs, size_t n, uint32_t flags, const TuneChoice *tc,
                           hwc_batch **out)
{
    return batch_create_impl(jobs, n, flags | HWC_FLAG_NO_TUNE, 1, out, tc);
}

extern "C" int hwc_batch_create(const hwc_job_t *jobs, size_t n_jobs, uint32_t flags, hwc_batch_t **out)
{
    if (!out) return set_error(HWC_ERR_ARG, "out is NULL");
    return batch_create_impl(jobs, n_jobs, flags, 1, out);
}

extern "C" int hwc_batch_launch(hwc_batch_t *b, void *stream)
{
    if (!b) return set_error(HWC_ERR_ARG, "batch is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    if (b->gexec) {
        HWC_CUDA_TRY(cudaGraphLaunch(b->gexec, s));
    } else {
        int rc = batch_enqueue(b, s, false);
        if (rc) return rc;
    }
    HWC_CUDA_TRY(cudaEventRecord(b->done, s));
    b->launched = true;
    return HWC_OK;
}

extern "C" int hwc_batch_result(hwc_batch_t *b, size_t i, hwc_hist_t **out)
{
    if (!b || !out) return set_error(HWC_ERR_ARG, "null argument");
    return batch_result_impl(b, i, out);
}

extern "C" int hwc_batch_kernel_launches(const hwc_batch_t *b, uint32_t *n)
{
    if (!b || !n) return set_error(HWC_ERR_ARG, "null argument");
    *n = b->launches_per_run;
    return HWC_OK;
}

extern "C" int hwc_batch_job_method(const hwc_batch_t *b, size_t i, uint32_t *method)
{
    if (!b || !method) return set_error(HWC_ERR_ARG, "null argument");
    if (i >= b->pos.size()) return set_error(HWC_ERR_RANGE, "job %zu of %zu", i, b->pos.size());
    const KJob &kj = b->jobs[b->pos[i]].kj;
    *method = (kj.method == 0 && kj.cls_n) ? 3u : kj.method;   // 3: the class-sharing variant
    return HWC_OK;
}

extern "C" int hwc_batch_io_bytes(const hwc_batch_t *b, uint64_t *h2d, uint64_t *d2h)
{
    if (!b) return set_error(HWC_ERR_ARG, "batch is NULL");
    if (h2d) *h2d = b->jobs.size() * sizeof(KJob) + b->n_starts * sizeof(uint64_t);
    if (d2h) *d2h = b->d2h_last;
    return HWC_OK;
}

extern "C" int hwc_batch_kernel_ms(hwc_batch_t *b, float *ms)
{
    if (!b || !ms) return set_error(HWC_ERR_ARG, "null argument");
    if (!b->t0) return set_error(HWC_ERR_STATE, "batch created without HWC_FLAG_TIMING");
    if (!b->launched) return set_error(HWC_ERR_STATE, "batch was not launched");
    HWC_CUDA_TRY(cudaEventSynchronize(b->done));
    HWC_CUDA_TRY(cudaEventElapsedTime(ms, b->t0, b->t1));
    return HWC_OK;
}

extern "C" void hwc_batch_free(hwc_batch_t *b)
{
    if (b && b->launched) cudaEventSynchronize(b->done);
    batch_release(b);
}

extern "C" int hwc_batch_run(const hwc_job_t *jobs, size_t n_jobs, uint32_t flags, void *stream,
                             hwc_hist_t **outs)
{
    if (!outs) return set_error(HWC_ERR_ARG, "outs is NULL");
    for (size_t i = 0; i < n_jobs; ++i) outs[i] = nullptr;
    hwc_batch *b = nullptr;
    int rc = HWC_OK;
    for (uint32_t scale = 1; scale <= 64; scale *= 8) {
        rc = batch_create_impl(jobs, n_jobs, flags, scale, &b);
        if (rc) return rc;
        rc = hwc_batch_launch(b, stream);
        for (size_t i = 0; rc == HWC_OK && i < n_jobs; ++i) rc = batch_result_impl(b, i, &outs[i]);
        hwc_batch_free(b);
        if (rc != HWC_ERR_TOO_LARGE) break;
        for (size_t i = 0; i < n_jobs; ++i) { hwc_hist_free(outs[i]); outs[i] = nullptr; }
    }
    if (rc) {
        for (size_t i = 0; i < n_jobs; ++i) { hwc_hist_free(outs[i]); outs[i] = nullptr; }
    }
    return rc;
}

// ---------------------------------------------------------------------
// single job

extern "C" int hwc_family_size(uint32_t q, const hwc_family_t *fam, uint64_t *n)
{
    if (!n) return set_error(HWC_ERR_ARG, "n is NULL");
    return family_size(q, fam, n);
}

extern "C" int hwc_count(uint32_t g, uint32_t q, const hwc_family_t *fam, uint64_t first,
                         uint64_t count, uint32_t flags, void *stream, hwc_hist_t **out)
{
    if (!out || !fam) return set_error(HWC_ERR_ARG, "null argument");
    *out = nullptr;
    hwc_job_t j{};
    j.g = g;
    j.q = q;
    j.family = *fam;
    j.first = first;
    j.count = count;
    return hwc_batch_run(&j, 1, flags | HWC_FLAG_PLAIN, stream, out);
}

extern "C" int hwc_count_members(uint32_t g, uint32_t q, const hwc_family_t *fam, uint64_t first,
                                 uint64_t count, int unfiltered, uint32_t flags, void *stream,
                                 int32_t *counts, uint8_t *sqf)
{
    if (!fam || (count && (!counts || !sqf))) return set_error(HWC_ERR_ARG, "null argument");
    hwc_job_t j{};
    j.g = g;
    j.q = q;
    j.family = *fam;
    j.first = first;
    j.count = count;
    uint64_t fam_n = 0;
    int rc = validate_job(j, &fam_n);
    if (rc) return rc;
    rc = prepare_count_kernels();
    if (rc) return rc;
    KJob kj;
    rc = fill_kjob(j, kj, &fam_n, (flags & (HWC_FLAG_HORNER | HWC_FLAG_FAN1 | HWC_FLAG_ALL_POINTS)) | kFlagNoWeights);
    if (rc) return rc;
    if (count == 0) return HWC_OK;
    kj.unfiltered = unfiltered ? 1u : 0u;
    cudaStream_t s = (cudaStream_t)stream;
    hwc_batch *b = new hwc_batch();   // allocation holder only
    LaunchShape sh;
    uint32_t launch_smem = kj.smem_bytes;
    if (kj.method == 2) {
        const Fan2Need need{kj.warp_off, kj.warp_bytes};
        rc = choose_shape_fan2((int)kj.d, &need, 1, &sh, &launch_smem);
        if (rc == HWC_OK) {
            rc = dalloc(b, &kj.wkeys, (uint64_t)sh.grid * (sh.block / 32) * kj.q * kj.q);
            kj.wkeys_stride = kj.q * kj.q;
        }
    } else {
        rc = choose_shape((int)kj.d, kj.method, kj.words, kj.smem_bytes, true, &sh);
    }
    uint64_t starts[2] = {0, 0};
    starts[1] = (kj.n_tiles + sh.item_tiles - 1) / sh.item_tiles;
    if (rc == HWC_OK &&
        ((rc = dalloc(b, &kj.member_counts, count * g)) || (rc = dalloc(b, &kj.member_sqf, count)) ||
         (rc = dalloc(b, &kj.stats, 4)) || (rc = dalloc(b, &b->d_jobs, 1)) ||
         (rc = dalloc(b, &b->d_item_start, 2)) || (rc = dalloc(b, &b->d_counters, 1)))) {
        batch_release(b);
        return rc;
    }
    if (rc) {
        batch_release(b);
        return rc;
    }
    cudaError_t ce = cudaMemsetAsync(kj.stats, 0, 4 * sizeof(unsigned long long), s);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(b->d_counters, 0, sizeof(unsigned long long), s);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(b->d_jobs, &kj, sizeof kj, cudaMemcpyHostToDevice, s);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(b->d_item_start, starts, sizeof starts, cudaMemcpyHostToDevice, s);
    if (ce != cudaSuccess) {
        batch_release(b);
        return set_error(HWC_ERR_CUDA, "setup: %s", cudaGetErrorString(ce));
    }
    rc = launch_persistent((int)kj.d, kj.method, kj.words, b->d_jobs, b->d_item_start, 1, starts[1],
                           b->d_counters, launch_smem, sh, s);
    if (rc == HWC_OK) {
        ce = cudaMemcpyAsync(counts, kj.member_counts, count * g * sizeof(int32_t), cudaMemcpyDeviceToHost, s);
        if (ce == cudaSuccess) ce = cudaMemcpyAsync(sqf, kj.member_sqf, count, cudaMemcpyDeviceToHost, s);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
        if (ce != cudaSuccess) rc = set_error(HWC_ERR_CUDA, "per-member run: %s", cudaGetErrorString(ce));
    }
    batch_release(b);
    return rc;
}

// ---------------------------------------------------------------------
// histogram ABI

extern "C" int hwc_hist_size(const hwc_hist_t *h, uint64_t *n_entries, uint64_t *n_squarefree,
                             uint64_t *n_total)
{
    if (!h) return set_error(HWC_ERR_ARG, "histogram is NULL");
    if (n_entries) *n_entries = h->mult.size();
    if (n_squarefree) *n_squarefree = h->n_sqf;
    if (n_total) *n_total = h->n_total;
    return HWC_OK;
}

extern "C" int hwc_hist_genus(const hwc_hist_t *h, uint32_t *g)
{
    if (!h || !g) return set_error(HWC_ERR_ARG, "null argument");
    *g = h->g;
    return HWC_OK;
}

extern "C" int hwc_hist_read(const hwc_hist_t *h, int32_t *counts, uint64_t *mult)
{
    if (!h) return set_error(HWC_ERR_ARG, "histogram is NULL");
    if (counts && !h->counts.empty()) std::memcpy(counts, h->counts.data(), h->counts.size() * sizeof(int32_t));
    if (mult && !h->mult.empty()) std::memcpy(mult, h->mult.data(), h->mult.size() * sizeof(uint64_t));
    return HWC_OK;
}

extern "C" int hwc_hist_merge(hwc_hist_t *into, const hwc_hist_t *from)
{
    if (!into || !from) return set_error(HWC_ERR_ARG, "histogram is NULL");
    if (into->g != from->g) return set_error(HWC_ERR_ARG, "genus mismatch %u vs %u", into->g, from->g);
    if (into->has_lam != from->has_lam)
        return set_error(HWC_ERR_ARG, "one histogram has factorisation patterns, the other not");
    const uint32_t g = into->g;
    HistMap m;
    for (const hwc_hist *h : {(const hwc_hist *)into, from})
        for (size_t i = 0; i < h->mult.size(); ++i)
            m[{h->has_lam ? h->lam[i] : 0ull, std::vector<int32_t>(&h->counts[i * g], &h->counts[i * g] + g)}] +=
                h->mult[i];
    hwc_hist *r = hist_from_map(g, m, into->n_total + from->n_total, into->has_lam);
    std::swap(*into, *r);
    delete r;
    return HWC_OK;
}

extern "C" int hwc_hist_from_arrays(uint32_t g, uint64_t n_entries, const int32_t *counts,
                                    const uint64_t *mult, uint64_t n_total, hwc_hist_t **out)
{
    if (!out || (n_entries && (!counts || !mult)) || g < 1 || g > (uint32_t)kMaxG)
        return set_error(HWC_ERR_ARG, "bad argument");
    HistMap m;
    for (uint64_t i = 0; i < n_entries; ++i)
        m[{0ull, std::vector<int32_t>(counts + i * g, counts + i * g + g)}] += mult[i];
    *out = hist_from_map(g, m, n_total, false);
    return HWC_OK;
}

// checkpoint file: "HWCH", version 1, g, flags (1: patterns, 2: job), n, n_total,
// n_squarefree, [job], then per entry counts[g] (i32), mult (u64), [pattern (u64)];
// every field little endian (the layout of the host; both hosts of this
// library are little endian)
namespace {
constexpr uint32_t kCkptMagic = 0x48435748u;   // "HWCH"
}

extern "C" int hwc_hist_save(const hwc_hist_t *h, const hwc_job_t *job, const char *path)
{
    if (!h || !path) return set_error(HWC_ERR_ARG, "null argument");
    FILE *f = std::fopen(path, "wb");
    if (!f) return set_error(HWC_ERR_ARG, "cannot open %s for writing", path);
    const uint64_t n = h->mult.size();
    const uint32_t head[4] = {kCkptMagic, 1u, h->g, (h->has_lam ? 1u : 0u) | (job ? 2u : 0u)};
    const uint64_t sizes[3] = {n, h->n_total, h->n_sqf};
    bool ok = std::fwrite(head, sizeof head, 1, f) == 1 && std::fwrite(sizes, sizeof sizes, 1, f) == 1;
    if (ok && job) ok = std::fwrite(job, sizeof *job, 1, f) == 1;
    for (uint64_t i = 0; ok && i < n; ++i) {
        ok = std::fwrite(&h->counts[i * h->g], sizeof(int32_t), h->g, f) == h->g &&
             std::fwrite(&h->mult[i], sizeof(uint64_t), 1, f) == 1;
        if (ok && h->has_lam) ok = std::fwrite(&h->lam[i], sizeof(uint64_t), 1, f) == 1;
    }
    ok = (std::fclose(f) == 0) && ok;
    return ok ? HWC_OK : set_error(HWC_ERR_ARG, "writing %s failed", path);
}

extern "C" int hwc_hist_load(const char *path, hwc_hist_t **out, hwc_job_t *job)
{
    if (!path || !out) return set_error(HWC_ERR_ARG, "null argument");
    *out = nullptr;
    if (job) std::memset(job, 0, sizeof *job);
    FILE *f = std::fopen(path, "rb");
    if (!f) return set_error(HWC_ERR_ARG, "cannot open %s", path);
    uint32_t head[4];
    uint64_t sizes[3];
    hwc_job_t jb{};
    bool ok = std::fread(head, sizeof head, 1, f) == 1 && head[0] == kCkptMagic && head[1] == 1u &&
              head[2] >= 1 && head[2] <= (uint32_t)kMaxG && std::fread(sizes, sizeof sizes, 1, f) == 1;
    if (ok && (head[3] & 2u)) ok = std::fread(&jb, sizeof jb, 1, f) == 1;
    hwc_hist *h = ok ? new hwc_hist() : nullptr;
    if (ok) {
        h->g = head[2];
        h->has_lam = head[3] & 1u;
        h->n_total = sizes[1];
        const uint64_t n = sizes[0];
        if (n > (1ull << 40)) ok = false;
        for (uint64_t i = 0; ok && i < n; ++i) {
            int32_t c[kMaxG];
            uint64_t m = 0, l = 0;
            ok = std::fread(c, sizeof(int32_t), h->g, f) == h->g && std::fread(&m, sizeof m, 1, f) == 1;
            if (ok && h->has_lam) ok = std::fread(&l, sizeof l, 1, f) == 1;
            if (!ok) break;
            h->counts.insert(h->counts.end(), c, c + h->g);
            h->mult.push_back(m);
            if (h->has_lam) h->lam.push_back(l);
            h->n_sqf += m;
        }
        ok = ok && h->n_sqf == sizes[2];
    }
    std::fclose(f);
    if (!ok) {
        delete h;
        return set_error(HWC_ERR_ARG, "%s is not a valid histogram checkpoint", path);
    }
    if (job && (head[3] & 2u)) *job = jb;
    *out = h;
    return HWC_OK;
}

extern "C" int hwc_hist_lambda(const hwc_hist_t *h, uint64_t *codes)
{
    if (!h) return set_error(HWC_ERR_ARG, "histogram is NULL");
    if (!h->has_lam) return set_error(HWC_ERR_STATE, "histogram counted without HWC_FLAG_LAMBDA");
    if (codes && !h->lam.empty()) std::memcpy(codes, h->lam.data(), h->lam.size() * sizeof(uint64_t));
    return HWC_OK;
}

extern "C" void hwc_hist_free(hwc_hist_t *h)
{
    delete h;
}

extern "C" const char *hwc_last_error(void)
{
    return hwc::g_err.c_str();
}

extern "C" const char *hwc_version(void)
{
    return "hwc 0.1 sm_103a";
}
