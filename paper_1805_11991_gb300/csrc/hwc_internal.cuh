// hwc_internal.cuh -- internal types of libhwc (not part of the C ABI).
//
// Element encoding (eq. 3.1): a nonzero element alpha^i of F_Q is stored as
// its log i in [0, L), L = Q - 1; zero is stored as L.  L is even because q
// is odd, so the quadratic character of alpha^i is (-1)^i (Sec. 1.1, chi).
#pragma once

#include <cstdint>
#include <cstddef>
#include <string>
#include <vector>
#include <mutex>
#include <cuda_runtime.h>

#include "../../include/hwc.h"

namespace hwc {

constexpr int kMaxG = 4;
constexpr int kMaxD = 2 * kMaxG + 2;        // degree 2g+2
constexpr int kMaxN = 16;                   // degree of F_Q over F_p (Q <= 2^24)
constexpr int kMaxE = 8;                    // degree of F_q over F_p
constexpr uint32_t kWideTable = 0xFFFFFFFFu; // table read from global memory
constexpr unsigned long long kEmptyKey = ~0ull;
constexpr int kTileMembers = 32;            // members per warp tile

// ---------------------------------------------------------------------
// errors (thread-local message, see hwc_last_error)
int set_error(int code, const char *fmt, ...);
#define HWC_CUDA_TRY(expr)                                                     \
    do {                                                                       \
        cudaError_t _e = (expr);                                               \
        if (_e != cudaSuccess)                                                 \
            return ::hwc::set_error(HWC_ERR_CUDA, "%s failed: %s (%s:%d)",     \
                                    #expr, cudaGetErrorString(_e), __FILE__,   \
                                    __LINE__);                                 \
    } while (0)

// ---------------------------------------------------------------------
// field tables of F_Q, Q = q^k, resident on one device
struct Tables {
    uint32_t q = 0, k = 0, p = 0, e = 0, n = 0, Q = 0, L = 0;
    uint32_t M[kMaxN + 1] = {};     // primitive modulus over F_p, M[n] = 1
    uint32_t mq[kMaxE + 1] = {};    // digit-convention modulus of F_q
    int device = -1;
    uint32_t *d_antilog = nullptr;  // [L]
    uint32_t *d_log = nullptr;      // [Q]
    uint32_t *d_zech = nullptr;     // [L], Z[L/2] = L
    uint32_t *d_coef_log = nullptr; // [q]
    // Zech table in the layout the count kernels read: entry u in [0, 2L)
    // is Z[u mod L], with the "1 + alpha^u = 0" entry replaced by the poison
    // value 2L, and entry 2L = 2L (absorbing).  u16 when 2L < 65536.
    uint16_t *d_zech2 = nullptr;    // [2L+1] or null
    uint32_t *d_zech2w = nullptr;   // [2L+1]
    // tripled layout: entry u in [0, 3L) is Z[u mod L] (poison 3L), T[3L] = 3L;
    // a step index z + d + j with z, d, j < L needs no reduction.  u16 when
    // 3L < 65536.
    uint16_t *d_zech3 = nullptr;    // [3L+1] or null
    // 17-bit layout for fields too large for u16 entries (2L >= 65536, L < 2^17 - 1):
    // entry u in [0, L] is lo[u] | (bit u of hi) << 16; Z[u] for u < L, and the
    // marker 0x1FFFF at u = L/2 (1 + alpha^u = 0) and at u = L (the poison of the
    // doubled index range folded back by one subtraction of L)
    uint16_t *d_z17lo = nullptr;    // [L+1] or null
    uint32_t *d_z17hi = nullptr;    // [(L+32)/32] or null
    // Fan-out rows (q <= 63): bit c of row l is 1 iff chi(alpha^l + c) = -1 for
    // the F_q digit c; the top bit (31 or 63) marks rows with alpha^l in F_q^x,
    // where alpha^l + c = 0 for the digit c = zdig[l / (L/(q-1))].
    uint32_t *d_rows32 = nullptr;   // [L + 1] when q <= 31; row L is y = 0
    unsigned long long *d_rows64 = nullptr;   // [L + 1] when q <= 63
    uint8_t *d_zdig = nullptr;      // [q]
    // F_q arithmetic on digits (k = 1, q <= 63): a*b, a-b (u8 [q*q]), 1/a (u8 [q])
    uint8_t *d_fq_mul = nullptr;
    uint8_t *d_fq_sub = nullptr;
    uint8_t *d_fq_inv = nullptr;
    // coordinates of F_{q^2} over F_q in the basis {1, alpha} (k = 2, q <= 31),
    // for alpha^l = e_y0 + e_y1 alpha: bits 0-7 -y0, bits 8-15 -y1; bits 16-23
    // 1/y1 and bits 24-31 -y0/y1 when y1 != 0, else 0 and -y0 (digits)
    uint32_t *d_coord2 = nullptr;   // [L]
    // Frobenius orbits (k >= 2): the logs j of one element alpha^j per orbit
    // {x, x^q, ..., x^(q^(k-1))} of the elements of exact degree k over F_q
    // (the smallest j of the orbit), ascending; n_reps of them
    uint32_t *d_reps = nullptr;     // [n_reps] or null (k = 1)
    uint32_t n_reps = 0;
};

// where a count kernel reads the Zech table of one field
enum TabKind : uint32_t {
    kTabTripleSmem = 0,   // d_zech3 staged in shared memory
    kTabDoubleSmem = 1,   // d_zech2 staged in shared memory
    kTabDoubleGlobal = 2, // d_zech2w read from global memory (L1/L2)
    kTab17Smem = 3,       // d_z17lo / d_z17hi staged in shared memory (per-member kernel)
};

int tables_build(uint32_t q, uint32_t k, Tables **out, uint64_t max_q = HWC_MAX_Q);
// one point per Frobenius orbit of the elements of exact degree k (host)
std::vector<uint32_t> orbit_reps(uint32_t q, uint32_t k, uint32_t L);
void tables_destroy(Tables *t);
// process-wide cache of tables per (device, q, k); never freed before exit
int tables_cached(uint32_t q, uint32_t k, const Tables **out, uint64_t max_q = HWC_MAX_Q);

// factor q = p^e, p odd prime
bool prime_power(uint32_t q, uint32_t *p, uint32_t *e);

// ---------------------------------------------------------------------
// device job descriptor (plain struct copied to device memory)
struct KJob {
    uint32_t g, q, d, kind;
    uint32_t p, unfiltered, pad0, pad1;
    uint64_t seed, first, count;
    uint64_t fam_mz;                  // q^(d-1): size of the MONIC_NOSUB family
    uint64_t qd;                      // q^d (ALL_DEG decode)
    uint64_t n_tiles;                 // ceil(count / 32)
    uint32_t Q[kMaxG], L[kMaxG];
    uint32_t barrett[kMaxG];          // floor(2^32 / L)
    uint32_t tab_off[kMaxG];          // u16 offset of the table in smem (smem kinds)
    uint32_t tab_kind[kMaxG];         // TabKind
    uint32_t tab_pad[kMaxG];          // 1: smem table padded by one u32 word per 32 (TabP)
    uint32_t coef_off[kMaxG];         // u32 offset of coef_log in smem (after tables)
    const uint16_t *zech3[kMaxG];
    const uint16_t *zech2[kMaxG];
    const uint32_t *zech2w[kMaxG];
    const uint32_t *coef_log[kMaxG];
    const uint16_t *z17lo[kMaxG];     // 17-bit layout (Tables::d_z17lo / d_z17hi) or null
    const uint32_t *z17hi[kMaxG];
    uint32_t tab_hi_off[kMaxG];       // kTab17Smem: u16 offset of the high-bit plane in smem
    // points evaluated in field m = k+1: one per Frobenius orbit of the
    // elements of exact degree m (reps[k], npts[k] of them), or every point of
    // F_Q^x (reps[k] null, npts[k] = L); field 1 always takes every point
    const uint32_t *reps[kMaxG];
    uint32_t npts[kMaxG];
    uint32_t zshift[kMaxG];           // two-level kernel: zeros ride in bits zshift.. of its
                                      // accumulators (0: field's zeros not needed apart)
    // HWC_FLAG_LAMBDA (per-member kernel): key = sum_k (a_k + key_bias[k]) << key_shift[k]
    // | (n_1..n_g in 4 bits each, then one bit: two factors of degree g+1) << lam_shift
    uint32_t lam_mode;
    uint32_t key_shift[kMaxG];
    int32_t key_bias[kMaxG];
    uint32_t lam_shift;
    // HWC_FAM_REDUCED: patterns A, B, (i, j) in index order (red_n of them),
    // red_start[] their first member index (red_start[red_n] = family size),
    // red_i / red_j the pattern (A: i = 0xFF, B: i = 0xFE), red_gcd, red_mult
    // the weight, red_w[t] the digit w^t
    static constexpr int kMaxPat = 2 + (2 * kMaxG) * (2 * kMaxG + 1) / 2;
    uint32_t red_n;
    uint64_t red_start[kMaxPat + 1];
    uint8_t red_i[kMaxPat], red_j[kMaxPat], red_gcd[kMaxPat];
    uint64_t red_mult[kMaxPat];
    uint32_t red_w[2 * kMaxG];
    uint32_t smem_u16;                // u16 words of zech2 tables staged in smem
    uint32_t smem_bytes;              // total dynamic smem for this job
    // c_0 fan-out (method 1): groups of q members that differ only in c_0
    uint32_t method;                  // 0 Horner tiles of 32 members, 1 fan-out groups of q,
                                      // 2 two-level fan-out groups of q^2
    uint32_t words;                   // method 1: row words, 1 (q <= 31) or 2 (q <= 63);
                                      // method 2: 1, or 2 for the weighted variant (mweight)
    uint64_t first_group;             // group of member `first`
    const void *rows[kMaxG];          // d_rows32 / d_rows64
    const uint8_t *zdig[kMaxG];
    uint32_t row_off[kMaxG];          // byte offset of the rows in smem
    uint32_t row16[kMaxG];            // method 2: 1 = the field's rows staged as int16 (q <= 15, bit 15 the flag)
    uint32_t zdig_off[kMaxG];         // byte offset of zdig in smem
    uint32_t zdiv[kMaxG];             // ceil(2^32 / (L/(q-1))): l / s by a high multiply
    uint32_t warp_off, warp_bytes;    // per-warp scratch in smem (method 2)
    uint32_t dense_off;               // method 2, g <= 2: smem offset of the CTA's (a_1, a_2) counters; 0: none
    uint32_t dense_w2, dense_n;       //   counter (a_1 + B_1) * w2 + (a_2 + B_2), n counters
    int32_t dense_b1, dense_b2;       //   Hasse-Weil bounds B_k = floor(2 g sqrt(q^k)) (B_2 = 0 for g = 1)
    unsigned long long *wkeys;        // per-warp member keys in global memory (method 2):
    uint32_t wkeys_stride, pad3;      //   slot blockIdx.x * warps + warp, stride q^2
    const uint8_t *fq_mul, *fq_sub, *fq_inv;   // digit arithmetic of F_q (fan-out jobs)
    uint32_t fq_off;                  // byte offset of mul | sub | inv | add in smem
    const uint32_t *coord2;           // method 2, g = 2: coordinates of F_{q^2} (Tables::d_coord2)
    uint32_t coord_off, pad4;         // byte offset of coord2 in smem; 0: not staged
    // outputs
    unsigned long long *hkeys;        // [hmask+1]
    unsigned long long *hcounts;      // [hmask+1]
    uint32_t hmask, pad2;
    unsigned long long *stats;        // [0] examined, [1] square-free, [2] overflow
    int32_t *member_counts;           // per-member mode: [count*g]
    uint8_t *member_sqf;              // per-member mode: [count]
    unsigned long long *out_keys;     // compacted histogram [hmask+1]
    unsigned long long *out_counts;
    unsigned long long *n_out;        // number of compacted entries
    // sampled family counted by the two-level kernel over the whole family:
    // mweight[i] = how often member i of HWC_FAM_MONIC_NOSUB was drawn by the
    // samples [s_first, s_first + s_count) (launch_sample_weights); the kernel
    // counts member i with that weight (0: not drawn).  first / count then
    // cover the whole family, or the window of HWC_FAM_MONIC_NOSUB_SAMPLED_WINDOW.
    // Null: every member in range has weight 1.
    uint32_t *mweight;
    uint64_t s_first, s_count;
    uint64_t w_first, w_n;            // mweight[i - w_first] for members w_first <= i < w_first + w_n
    // class-sharing kernel (method 0 with words = 1, classes.cuh): the samples
    // sorted by class c = (c_2..c_{d-2}) before the count (launch_class_sort);
    // cls_sorted holds c_0 + c_1 q of each sample, grouped by class;
    // cls_cnt[c] = end of class c in cls_sorted after the sort;
    // cls_tiles[t] = (class, start) of up to 32 samples, class 0xFFFFFFFF past
    // the last tile (n_tiles is the bound ceil(count / 32) + cls_n)
    uint2 *cls_tiles;
    uint32_t *cls_cnt;
    uint32_t *cls_sorted;
    uint32_t cls_n;                   // classes: q^(d-3)
};

// launch helpers (count_kernels.cu)
struct LaunchShape {
    int block = 256;       // threads per CTA (multiple of 32)
    int grid = 0;          // CTAs (0 = derive)
    int item_tiles = 4;    // tiles per queue item (persistent)
};
int launch_clear(const KJob *d_jobs, uint32_t n_jobs, unsigned long long *d_counters,
                 uint32_t n_counters, cudaStream_t s);
// one persistent launch over jobs of one degree, method and row width
int launch_persistent(int D, uint32_t method, uint32_t words, const KJob *d_jobs,
                      const uint64_t *d_item_start, uint32_t n_jobs, uint64_t n_items,
                      unsigned long long *d_counter, uint32_t max_smem, const LaunchShape &sh,
                      cudaStream_t s);
int launch_compact(const KJob *d_jobs, uint32_t n_jobs, cudaStream_t s);
// the multiplicities kj.mweight of a sampled job counted by the two-level
// kernel: cleared, then one atomic add per sample (stream-ordered)
int launch_sample_weights(const KJob &kj, cudaStream_t s);
// sort the samples of a class-sharing job by class (no-op for other jobs)
int launch_class_sort(const KJob &kj, cudaStream_t s);
// raise the dynamic shared memory limit of the count kernels (once per device)
int prepare_count_kernels(void);
int max_ctas_per_sm(int D, uint32_t method, uint32_t words, int block, uint32_t smem_bytes,
                    bool persistent, int *out);
int device_sm_count(void);
uint32_t device_smem_optin(void);

// fills the job's smem layout (tab_off, coef_off, row_off, smem_bytes)
// A kernel choice for one class of jobs (g, q, degree, family kind), made by
// the autotuner (tune.cu) or left to the default rule.
struct TuneChoice {
    int method = -1;          // -1: default rule; 0 per member, 1 c_0 fan-out, 2 (c_1, c_0) fan-out
    int warps = 0;            // two-level kernel: warps per CTA (0: the most resident)
    bool no_triple = false;   // shared Zech tables in the doubled layout only
};
bool layout_job_smem(KJob &j, uint32_t smem_limit, bool no_triple = false);
// a sampled job counted by the two-level kernel over its whole family, with
// the samples' multiplicities as weights (KJob::mweight)
inline bool needs_weights(const KJob &kj)
{
    return (kj.kind == HWC_FAM_MONIC_NOSUB_SAMPLED || kj.kind == HWC_FAM_MONIC_NOSUB_SAMPLED_WINDOW) && kj.method == 2;
}
// fill_kjob flag (internal): keep sampled families on the per-member kernel
// (per-sample outputs need the members in sample order)
constexpr uint32_t kFlagNoWeights = 1u << 31;
// fill_kjob flag (internal): no class-sharing kernel (the server's requests
// are slices too small to share chains)
constexpr uint32_t kFlagNoClass = 1u << 30;
// the class-sharing kernel needs this many samples per class on average
constexpr uint64_t kClsMinPerClass = 16;
constexpr uint32_t kClsWarpBytes = 512;   // class-sharing kernel: per-warp staging of 64 (log u, log x)
constexpr uint32_t kClsMaxWarps = 24;
// the points field k (1-based) evaluates: one per Frobenius orbit (orbits,
// k >= 2) or all of F_Q^x; and the two-level kernel's zero shift
void set_points(KJob &kj, uint32_t k, const Tables *t, bool orbits);
// validates a job and fills a KJob (tables, method, layout); outputs left null
int fill_kjob(const hwc_job_t &jb, KJob &kj, uint64_t *fam_n, uint32_t flags, const TuneChoice *tc = nullptr);
// autotuner: the fastest measured choice for the job's class (measured on a
// probe slice the first time a class is seen, then cached per process and,
// with HWC_TUNE_CACHE set, in that file); tune_lookup only reads the cache
int tune_choice(const hwc_job_t &jb, uint32_t flags, TuneChoice *out);
bool tune_lookup(const hwc_job_t &jb, uint32_t flags, TuneChoice *out);
// a batch whose jobs take the given choices (no autotuning); for probes
int batch_create_with(const hwc_job_t *jobs, size_t n, uint32_t flags, const TuneChoice *tc, hwc_batch **out);
// launch shape for a kernel (degree, method, row words) at this much dynamic smem
int choose_shape(int D, uint32_t method, uint32_t words, uint32_t smem, bool persistent, LaunchShape *out);
// kernel entry points by degree: which = 1 persistent (<= 256 threads),
// 2 allocation-free, 3 persistent with up to 768 threads
const void *horner_kernel(int D, int which);
const void *horner_kernel_a(int D, int which);   // horner_a.cu, D = 3..6
const void *horner_kernel_b(int D, int which);   // horner_b.cu, D = 7, 8
const void *horner_kernel_c(int D, int which);   // horner_c.cu, D = 9, 10
// class-sharing kernels (classes.cuh), D = 3..6: which = 1 (<= 256 threads) or 3 (<= 768)
const void *cls_kernel_a(int D, int which);   // cls_a.cu
// c_0 fan-out kernels (fanout.cuh), W = row words
const void *fan_kernel(int D, int W, bool persistent);
const void *fan_kernel_a(int D, int W, bool persistent);   // fanout_a.cu, D = 3, 4
const void *fan_kernel_b(int D, int W, bool persistent);   // fanout_b.cu, D = 5
const void *fan_kernel_c(int D, int W, bool persistent);   // fanout_c.cu, D = 6
const void *fan_kernel_d(int D, int W, bool persistent);   // fanout_d.cu, D = 7
const void *fan_kernel_f(int D, int W, bool persistent);   // fanout_f.cu, D = 8
// two-level fan-out kernels (fanout2.cuh), q <= 31
const void *fan2_kernel(int D, bool weighted);
const void *fan2_kernel_a(int D);   // fan2_a.cu, D = 3..6
const void *fan2_kernel_b(int D);   // fan2_b.cu, D = 7..10
const void *fan2_kernel_wa(int D);  // fan2_wa.cu, D = 3..6, members weighted by their draws
const void *fan2_kernel_wb(int D);  // fan2_wb.cu, D = 7..10
constexpr int kFan2WarpsHost = 4;   // warps per CTA of the two-level kernel
// Per-warp shared scratch of the two-level kernel for q (S = floor(32/q)
// lanes per value of c_1; offsets in bytes):
//   U[us] u32: staged log u(x) for 64 points; us = 96 when 64/S is not a
//              multiple of 8 (the lanes' 8-point blocks overrun 64), else 64
//   Dd[us] u32: staged log u(x) - log x (orbit points)
//   acc[32][q] u16: per-lane rows of 2 cnt + z for every c_0 (lane s q + b
//              holds (c_1 = b, chunk s); lanes past S q fill unused rows)
//   rq[kFan2Queue][32] u16: per-lane queue of row indices with a zero digit
//   sqf[ceil(q^2/32)] u32: square-free member bits
//   par[64] u32: the group's digits c_i, the field's logs lam_i and h chain
//   a1[q^2] u16 (dense histogram only): a_1 + 32768 of every member
constexpr uint32_t kFan2Queue = 14;   // drained once a lane holds more than 6 (a block adds up to 8)
// The two-level kernel stages each Zech table behind a prefix of 64 entries
// (the table continued periodically to negative indices) with the poison
// value 0xFFFF, and each fan-out row table as rows[i mod L] for i < L + 8
// followed by the row of y = 0 at L + 8.
constexpr uint32_t kFan2Prefix = 64;
constexpr uint32_t kFan2ZeroRow = 8;   // row index L + 8
struct Fan2Layout {
    uint32_t us, ds_off, acc_off, rq_off, sqf_off, par_off, a1_off, bytes;
};
__host__ __device__ inline Fan2Layout fan2_layout(uint32_t q, bool dense)
{
    Fan2Layout l;
    const uint32_t S = 32 / q, nw = (q * q + 31) / 32;
    l.us = (S == 1 || S == 2 || S == 4 || S == 8) ? 64 : 96;
    l.ds_off = 4 * l.us;
    l.acc_off = 8 * l.us;
    l.rq_off = l.acc_off + ((64 * q + 3) & ~3u);
    l.sqf_off = l.rq_off + 2 * kFan2Queue * 32;
    l.par_off = (l.sqf_off + 4 * nw + 15) & ~15u;
    l.a1_off = l.par_off + 4 * 64;
    l.bytes = (l.a1_off + (dense ? 2 * q * q : 0) + 15) & ~15u;
    return l;
}
inline uint32_t fan2_warp_bytes(uint32_t q, bool dense) { return fan2_layout(q, dense).bytes; }
// launch shape of the two-level kernel for jobs with these smem needs: the
// block (4, 8, 12, 16 or 24 warps) that keeps most warps resident; *smem receives the
// dynamic shared memory of that block
struct Fan2Need {
    uint32_t warp_off, warp_bytes;
};
int choose_shape_fan2(int D, const Fan2Need *needs, size_t n, LaunchShape *out, uint32_t *smem, int warps = 0);
const void *fan_kernel_e(int D, int W, bool persistent);   // fanout_e.cu, D = 9, 10
// hash slots for a job of `count` members (power of two)
uint32_t hash_capacity(uint32_t g, uint32_t q, uint64_t count, uint32_t scale);

}  // namespace hwc

// opaque ABI types
struct hwc_tables {
    hwc::Tables *t;
};

struct hwc_hist {
    uint32_t g = 0;
    std::vector<int32_t> counts;   // n * g, lexicographically sorted (after lam)
    std::vector<uint64_t> mult;
    std::vector<uint64_t> lam;     // factorisation pattern codes (HWC_FLAG_LAMBDA), else empty
    bool has_lam = false;
    uint64_t n_total = 0, n_sqf = 0;
};

namespace hwc {
// decode compacted (key, count) pairs into a sorted histogram
hwc_hist *hist_from_keys(const KJob &kj, const unsigned long long *keys,
                         const unsigned long long *cnt, uint64_t n, uint64_t n_total);
}  // namespace hwc
