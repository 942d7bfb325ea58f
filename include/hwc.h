/*
 * hwc.h -- C ABI of the GB300 point-counting library (libhwc.so).
 *
 * The library counts points on every hyperelliptic curve C_f : y^2 = f(x) of
 * genus g in a coefficient family over F_q, over every F_{q^k}, k = 1..g, and
 * returns the exact histogram of the tuples (#C_f(F_q), ..., #C_f(F_{q^g}))
 * over the square-free members f.  This is the inner part of Algorithm 1 of
 * Raum, "Hyperelliptic curves over small finite fields and GPU accelerators"
 * (arXiv:1805.11991): from the choice of f through the point counts, and the
 * histogram increment with weight 1.
 *
 * Conventions shared by every entry point
 *  - Return value: HWC_OK (0) or a negative HWC_ERR_* code.  Nothing throws
 *    across the ABI.  hwc_last_error() gives a message for the calling thread.
 *  - q is an odd prime power, 1 <= g <= 4, 1 <= k <= g, deg f = d in
 *    {2g+1, 2g+2} (Sec. 1.1).  Q = q^k must be at most HWC_MAX_Q.
 *  - F_q digits: an integer c in [0, q), c = sum_i b_i p^i, stands for
 *    sum_i b_i T^i in F_p[T]/m(T), m the first monic irreducible polynomial of
 *    degree e (q = p^e) in the order of the index sum_i m_i p^i.  So 0 and 1
 *    are the field's 0 and 1.  Coefficient c_i of f is digit i of the member
 *    index, base q, little endian (see hwc_family_t).
 *  - Handles (hwc_tables_t, hwc_hist_t, hwc_batch_t, hwc_server_t) are owned
 *    by the library and released with their *_free / *_close function.
 *    Device memory behind them is allocated by the library on the current
 *    CUDA device.
 *  - `stream` arguments are a cudaStream_t passed as void* (NULL = the
 *    default stream).
 */
#ifndef HWC_H
#define HWC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HWC_OK 0
#define HWC_ERR_ARG (-1)       /* bad q, g, k, degree, family or flags      */
#define HWC_ERR_RANGE (-2)     /* first + count beyond the family           */
#define HWC_ERR_TOO_LARGE (-3) /* Q above HWC_MAX_Q, or histogram overflow  */
#define HWC_ERR_NOMEM (-4)     /* device or host allocation failed          */
#define HWC_ERR_CUDA (-5)      /* a CUDA call failed (message has details)  */
#define HWC_ERR_TIMEOUT (-6)   /* a bounded wait ran out                    */
#define HWC_ERR_BUSY (-7)      /* server admission refused (no room)        */
#define HWC_ERR_STATE (-8)     /* call out of order (e.g. result not ready) */

#define HWC_MAX_Q 262144u      /* largest field size F_{q^k} accepted       */
#define HWC_MAX_G 4u

/* Families of f (Sec. 1.1, Algorithm 1).  Member idx decodes to
 * c_0..c_d by base-q digits of idx, little endian:
 *  HWC_FAM_ALL_DEG       exact degree d, any lead: c_i = digit i of
 *                        (idx mod q^d) for i < d, c_d = 1 + floor(idx / q^d);
 *                        (q-1) q^d members.
 *  HWC_FAM_MONIC_NOSUB   monic, c_{d-1} = 0, (c_0..c_{d-2}) = digits of idx;
 *                        q^(d-1) members.
 *  HWC_FAM_MONIC_NOSUB_SAMPLED
 *                        member j (0 <= j < sample_count) is member
 *                        floor(z_j * q^(d-1) / 2^64) of HWC_FAM_MONIC_NOSUB,
 *                        z_j the SplitMix64 output for state seed + (j+1) *
 *                        0x9E3779B97F4A7C15 (Steele, Lea, Flood 2014);
 *                        drawn with replacement. */
#define HWC_FAM_ALL_DEG 0u
#define HWC_FAM_MONIC_NOSUB 1u
#define HWC_FAM_MONIC_NOSUB_SAMPLED 2u
/*  HWC_FAM_REDUCED       the reduced polynomials P'_d of Sec. 1.2-1.3 (p not
 *                        dividing d): one polynomial per class of the affine
 *                        maps X -> aX + b and f -> f / e^2, with the first
 *                        coefficient below the lead set to 1 (the quadratic
 *                        twist folded in).  Patterns in this order:
 *                          A: c_d X^d + 1, B: c_d X^d + X (q-1 members each),
 *                          (i, j), 1 <= i <= d-2, 0 <= j < i (i outer):
 *                          c_d X^d + X^i + w^t X^j + c_{j-1} X^(j-1) + ... + c_0,
 *                          t < gcd(q-1, i-j), w the smallest digit generating
 *                          F_q^x; (q-1) gcd(q-1, i-j) q^j members, index =
 *                          c_0 + c_1 q + ... + q^j (t + gcd (c_d - 1)).
 *                        Each member is counted with weight mult(f) (q(q-1)/2
 *                        for A and B, q(q-1)^2 / (2 gcd(q-1, i-j)) for (i, j))
 *                        twice: with its own (a_1..a_g) and with its twist's,
 *                        a_k -> (-1)^k a_k.  The histogram then equals the one
 *                        over every square-free f of degree d (eq. 1.2). */
#define HWC_FAM_REDUCED 3u
/*  HWC_FAM_MONIC_NOSUB_SAMPLED_WINDOW
 *                        the draws of HWC_FAM_MONIC_NOSUB_SAMPLED (samples
 *                        0 <= j < sample_count, seed) that land in a window of
 *                        member indices: the job's [first, first + count)
 *                        names members of HWC_FAM_MONIC_NOSUB (q^(d-1) of
 *                        them), and each member of the window is counted as
 *                        often as the samples draw it.  Disjoint windows
 *                        covering the family add up to the whole sampled
 *                        family, which lets a request stream cut a densely
 *                        drawn family into pieces of equal work without
 *                        losing the whole-family kernel.  Only that kernel
 *                        runs it: q <= 31, sample_count >= q^(d-1) / 32 and
 *                        < 2^27, tables in shared memory; otherwise, and for
 *                        hwc_count_members, HWC_ERR_ARG.  No counterpart in
 *                        the paper (serving). */
#define HWC_FAM_MONIC_NOSUB_SAMPLED_WINDOW 4u

typedef struct {
    uint32_t kind;          /* HWC_FAM_*                                   */
    uint32_t degree;        /* d                                           */
    uint64_t seed;          /* sampled family only                         */
    uint64_t sample_count;  /* sampled family only                         */
} hwc_family_t;

/* One counting job: members [first, first + count) of a family. */
typedef struct {
    uint32_t g;
    uint32_t q;
    hwc_family_t family;
    uint64_t first;
    uint64_t count;
} hwc_job_t;

typedef struct hwc_tables hwc_tables_t;
typedef struct hwc_hist hwc_hist_t;
typedef struct hwc_batch hwc_batch_t;
typedef struct hwc_server hwc_server_t;

/* Message of the last failed call on this thread ("" if none). */
const char *hwc_last_error(void);

/* Library version string. */
const char *hwc_version(void);

/* ------------------------------------------------------------------ */
/* Field tables (Sec. 2.3, eq. 3.1-3.2)                                */

/* Build, on the current device, the Zech-logarithm tables of F_Q, Q = q^k:
 * a primitive element alpha (F_Q = F_p[X]/M(X), M the first primitive
 * polynomial of degree e*k over F_p by index, alpha = X), antilog[i] =
 * alpha^i, log (log of 0 = L = Q-1, the encoding of eq. 3.1), the Zech table
 * Z[n] = log(1 + alpha^n) with Z[L/2] = L (eq. 3.2), and the logs of the F_q
 * digits embedded in F_Q.  *out receives a library-owned handle; errors:
 * HWC_ERR_ARG (q not an odd prime power, k = 0), HWC_ERR_TOO_LARGE
 * (Q > HWC_MAX_Q), HWC_ERR_NOMEM, HWC_ERR_CUDA.  Synchronous. */
int hwc_field_tables(uint32_t q, uint32_t k, hwc_tables_t **out);

/* Facts about built tables.  info[0..] = q, k, p, e, Q, L, primitive-poly
 * degree n = e*k, then M_0..M_n (n+1 values), then the digit modulus
 * m_0..m_e (e+1 values).  `cap` is the length of info; returns the number
 * of values written, or a negative error. */
int hwc_tables_info(const hwc_tables_t *t, uint32_t *info, uint32_t cap);

/* Copy the tables to host arrays (any may be NULL): antilog[L] (element of
 * F_Q as the integer sum_i a_i p^i of its coefficients on 1, X, X^2, ...),
 * log[Q], zech[L], coef_log[q].  Synchronous. */
int hwc_tables_read(const hwc_tables_t *t, uint32_t *antilog, uint32_t *log,
                    uint32_t *zech, uint32_t *coef_log);

void hwc_tables_free(hwc_tables_t *t);

/* ------------------------------------------------------------------ */
/* Counting                                                            */

/* Number of members of a family over F_q into *n. */
int hwc_family_size(uint32_t q, const hwc_family_t *fam, uint64_t *n);

/* Flags for hwc_count / hwc_batch_create. */
#define HWC_FLAG_PLAIN 0x1u       /* one launch per job (no persistent queue)  */
#define HWC_FLAG_GRAPH 0x2u       /* capture the launch sequence in a CUDA graph */
#define HWC_FLAG_HORNER 0x4u      /* force the per-member Horner kernel        */
/* Kernels: enumerated families with q <= 31 use the two-level fan-out (q^2
 * members sharing c_2..c_d per warp), q <= 63 the one-level c_0 fan-out (q
 * members per warp), everything else (larger q, reduced families, sparse
 * samples) the per-member Horner kernel.  A sampled family with q <= 31 and
 * at least one sample per 32 members of HWC_FAM_MONIC_NOSUB (fewer than 2^27
 * samples) runs the two-level fan-out over the whole family, each member
 * weighted by how often the samples drew it (4 bytes of device memory per
 * member, cleared and filled in every run).  All give identical counts. */
#define HWC_FLAG_NO_TUNE 0x8u     /* skip the autotuner, use defaults          */
#define HWC_FLAG_TIMING 0x10u     /* time the count kernel(s) with CUDA events */
#define HWC_FLAG_FAN1 0x20u       /* one-level c_0 fan-out even where the
                                     two-level (c_1, c_0) kernel applies */
/* By default the kernels evaluate f at one point per Frobenius orbit: x and
 * x^q, x^(q^2), ... give the same chi(f(x)) because f has coefficients in
 * F_q, so F_{q^k} is covered by the elements of exact degree m | k, one per
 * orbit of m conjugates, each weighted by m (and chi_{q^k} = chi_{q^m}^(k/m)
 * on F_{q^m}).  The counts are the same as evaluating every point. */
#define HWC_FLAG_ALL_POINTS 0x40u /* evaluate every x of every F_{q^k} instead */
/* Key the histogram also by the factorisation pattern lambda(f) of eq. 1.2:
 * the partition of 2g+2 formed by the degrees of the irreducible factors of
 * f over F_q, with one more part 1 when deg f = 2g+1 (read the patterns with
 * hwc_hist_lambda).  The kernels get the factors of degree m <= g from the
 * zeros of f at the Frobenius-orbit points of exact degree m (one per
 * irreducible factor of degree m), the rest from the degree left over and,
 * when 2g+2 is left (one factor of degree 2g+2 or two of degree g+1), from
 * the quadratic character of the discriminant of f (Stickelberger: the
 * number of irreducible factors r of a square-free f has
 * (-1)^(deg f - r) = chi(disc f)).  Runs the per-member kernel; not with
 * HWC_FLAG_ALL_POINTS. */
#define HWC_FLAG_LAMBDA 0x80u

/* Histogram of (#C(F_q), ..., #C(F_{q^g})) over the square-free members
 * [first, first+count) of the family (Algorithm 1: point counts and the
 * histogram increment, every weight 1).  Synchronous on `stream`; *out receives a library-owned
 * histogram.  Errors: HWC_ERR_ARG, HWC_ERR_RANGE, HWC_ERR_TOO_LARGE,
 * HWC_ERR_NOMEM, HWC_ERR_CUDA. */
int hwc_count(uint32_t g, uint32_t q, const hwc_family_t *fam, uint64_t first,
              uint64_t count, uint32_t flags, void *stream, hwc_hist_t **out);

/* Per-member counts (for checking): counts[i*g + k-1] = #C(F_{q^k}) and
 * sqf[i] = 1 if member first+i is square-free.  With unfiltered = 0 the
 * counts of non-square-free members are 0; with unfiltered = 1 they are the
 * point-count formula applied anyway.  flags: 0, HWC_FLAG_HORNER (use the
 * per-member kernel everywhere) or HWC_FLAG_FAN1 (one-level fan-out where the
 * two-level kernel would apply).  `counts`
 * (count*g int32) and `sqf` (count bytes) are HOST arrays.  Synchronous. */
int hwc_count_members(uint32_t g, uint32_t q, const hwc_family_t *fam,
                      uint64_t first, uint64_t count, int unfiltered, uint32_t flags,
                      void *stream, int32_t *counts, uint8_t *sqf);

/* Histograms.  A histogram is the multiset of tuples (#C_1..#C_g), one per
 * square-free member, i.e. the map N_{g,q} of eq. 1.2 with every weight 1 and
 * the tuple keyed by #C_k = q^k + 1 - a_k (eq. 1.1) instead of a_k, without the
 * factorisation partition.  Histograms of disjoint member ranges add.
 *
 * Contents: n_entries distinct tuples; n_squarefree = sum of the
 * multiplicities; n_total = members examined. */
int hwc_hist_size(const hwc_hist_t *h, uint64_t *n_entries, uint64_t *n_squarefree,
                  uint64_t *n_total);
/* g of the histogram. */
int hwc_hist_genus(const hwc_hist_t *h, uint32_t *g);
/* Host arrays: counts[n_entries*g] (#C_1..#C_g per entry, sorted
 * lexicographically), mult[n_entries]. */
int hwc_hist_read(const hwc_hist_t *h, int32_t *counts, uint64_t *mult);
/* Factorisation patterns of a histogram counted with HWC_FLAG_LAMBDA:
 * codes[n_entries], entry i's lambda as sum_m n_m 16^(m-1), n_m the parts
 * equal to m (m = 1..2g+2).  Entries are then sorted by code, then by tuple.
 * HWC_ERR_STATE for a histogram without patterns. */
int hwc_hist_lambda(const hwc_hist_t *h, uint64_t *codes);
/* into += from (same g, both with or both without patterns); shards of one
 * family and resumed runs add up. */
int hwc_hist_merge(hwc_hist_t *into, const hwc_hist_t *from);
/* New histogram from host arrays (e.g. a checkpoint), same layout as read. */
int hwc_hist_from_arrays(uint32_t g, uint64_t n_entries, const int32_t *counts,
                         const uint64_t *mult, uint64_t n_total, hwc_hist_t **out);
void hwc_hist_free(hwc_hist_t *h);

/* Checkpoints.  A histogram is the count of a member range; ranges of one
 * job add (hwc_hist_merge), so an interrupted job resumes from its first
 * uncounted member.  hwc_hist_save writes the histogram (tuples,
 * multiplicities, patterns if any, members examined) and, when job is not
 * NULL, the job it counts (members [job->first, job->first + job->count)
 * done) to a little-endian binary file; hwc_hist_load reads it back, and
 * fills *job when job is not NULL and the file has one (else zeroes it).
 * Errors: HWC_ERR_ARG (bad file), HWC_ERR_NOMEM. */
int hwc_hist_save(const hwc_hist_t *h, const hwc_job_t *job, const char *path);
int hwc_hist_load(const char *path, hwc_hist_t **out, hwc_job_t *job);

/* ------------------------------------------------------------------ */
/* Batched execution: many jobs in one persistent launch               */
/* The paper launches one kernel per curve and field (Sec. 3.3); batching
 * many jobs of uneven size into one launch has no counterpart there.  Each
 * job's histogram is the one hwc_count gives for it alone. */

/* Prepare a batch: builds (or reuses) the field tables of every job,
 * allocates one device histogram per job and the work queue, and picks the
 * kernel parameters.  Unless HWC_FLAG_NO_TUNE, the autotuner times the
 * candidate choices for each class of jobs (g, q, degree, family kind) the
 * first time the class is seen, on a probe slice of that job (about two work
 * items per resident warp; smaller jobs keep the default rule): the kernel
 * (per-member evaluation, or fan-out over c_0 or (c_1, c_0)), the warps per
 * CTA and the layout of the shared Zech tables.  It launches probe kernels on
 * the legacy default stream before returning.  Choices are cached per
 * process, and in the file named by the environment variable HWC_TUNE_CACHE
 * when it is set.  Every choice gives the same histograms.  With
 * HWC_FLAG_PLAIN each job gets its own launch instead of one persistent
 * launch.  With HWC_FLAG_GRAPH the launch sequence is captured once in a
 * CUDA graph. */
int hwc_batch_create(const hwc_job_t *jobs, size_t n_jobs, uint32_t flags,
                     hwc_batch_t **out);
/* Enqueue one complete run of the batch on `stream` (asynchronous): clears
 * the histograms and the queue, then runs every job. */
int hwc_batch_launch(hwc_batch_t *b, void *stream);
/* Wait for the last launch, copy out and sort the histogram of job i. */
int hwc_batch_result(hwc_batch_t *b, size_t i, hwc_hist_t **out);
/* Number of kernel launches one hwc_batch_launch enqueues. */
int hwc_batch_kernel_launches(const hwc_batch_t *b, uint32_t *n);
/* Count kernel that job i of the batch runs: 0 per-member Horner evaluation
 * (Algorithm 1 as written), 1 fan-out over c_0 (groups of q members sharing
 * c_1..c_d), 2 fan-out over (c_1, c_0) (groups of q^2 members), 3 per-member
 * evaluation of a sampled family sorted by its high digits c_2..c_{d-2}
 * (degrees 3..6, at least 16 samples per class on average; the samples of a
 * class share the chain for u = sum_{i>=2} c_i x^i).  The choice
 * is made at hwc_batch_create from the family, q and the shared-memory room
 * of the field tables (HWC_FLAG_HORNER / HWC_FLAG_FAN1 restrict it). */
int hwc_batch_job_method(const hwc_batch_t *b, size_t i, uint32_t *method);
/* Bytes one hwc_batch_launch copies host->device (job descriptors, from
 * pinned memory) and hwc_batch_result copies device->host for all jobs of
 * the last launch (statistics plus the compacted histograms). */
int hwc_batch_io_bytes(const hwc_batch_t *b, uint64_t *h2d, uint64_t *d2h);
/* With HWC_FLAG_TIMING: device time in ms of the count kernel(s) of the last
 * launch (CUDA events on the launch stream), after waiting for it. */
int hwc_batch_kernel_ms(hwc_batch_t *b, float *ms);
void hwc_batch_free(hwc_batch_t *b);
/* Convenience: create, launch, wait, results for every job (outs[n_jobs]). */
int hwc_batch_run(const hwc_job_t *jobs, size_t n_jobs, uint32_t flags, void *stream,
                  hwc_hist_t **outs);

/* ------------------------------------------------------------------ */
/* Serving: a request loop with continuous batching                    */
/* No counterpart in the paper (its runs are offline).  Each request's
 * histogram is the one hwc_count gives for the same job alone. */

typedef struct {
    uint64_t device_bytes;   /* admission budget for tables + histograms    */
    uint32_t max_active;     /* jobs on the device at once                  */
    uint32_t step_items;     /* work per device step (0 = library default)  */
} hwc_server_config_t;

/* Start a server thread that keeps field tables resident and runs, step
 * after step, one batched launch over the active requests; requests that
 * arrive meanwhile join at the next step once memory and a slot are free. */
int hwc_serve_open(const hwc_server_config_t *cfg, hwc_server_t **out);
/* Queue a request; *ticket identifies it. */
int hwc_serve_submit(hwc_server_t *s, const hwc_job_t *job, uint64_t *ticket);
/* Non-blocking: HWC_OK with *out set when done, HWC_ERR_STATE if not yet.
 * timeout_ms > 0 waits at most that long. */
int hwc_serve_poll(hwc_server_t *s, uint64_t ticket, uint32_t timeout_ms,
                   hwc_hist_t **out);
/* Latency of a finished request: submit -> admitted -> done, microseconds. */
int hwc_serve_latency(hwc_server_t *s, uint64_t ticket, double *queued_us,
                      double *total_us);
/* Stop the thread (finishing the active step) and free everything. */
int hwc_serve_close(hwc_server_t *s);

/* ------------------------------------------------------------------ */
/* Single curves (Sec. 4, Table 1: one curve counted over F_{p^2})     */

#define HWC_MAX_Q_CURVE (1u << 24)   /* largest F_{q^k} for hwc_curve_count */

/* #C_f(F_{q^k}) of explicit curves y^2 = f_i(x), i < n: coeffs[i*(d+1) + j]
 * is the F_q digit c_j of f_i (c_d != 0), counts[i] receives
 * r^0 + 2 r^sq + 1 + chi(f(inf)) as in Sec. 1.1 (f need not be
 * square-free).  The points are spread over the whole GPU: every field
 * F_{q^m}, m | k, evaluates one point per Frobenius orbit of its elements of
 * exact degree m, with Zech tables of up to HWC_MAX_Q_CURVE elements read
 * from global memory (L2-resident); the tables are built on first use and
 * cached.  1 <= d <= 10; coeffs and counts are HOST arrays.  Synchronous on
 * `stream`.  Errors: HWC_ERR_ARG, HWC_ERR_TOO_LARGE (q^k above
 * HWC_MAX_Q_CURVE), HWC_ERR_NOMEM, HWC_ERR_CUDA.  If ms is not NULL it
 * receives the device time of the count kernels (CUDA events). */
int hwc_curve_count(uint32_t q, uint32_t k, uint32_t d, uint64_t n, const uint32_t *coeffs, int64_t *counts,
                    void *stream, float *ms);

/* ------------------------------------------------------------------ */
/* Counting without device allocation                                  */

/* Histogram of one job for callers that cannot allocate device memory when
 * they count: for example a process that reserves the device memory up front
 * and forbids further cudaMalloc, or a host thread that must not call
 * cudaMalloc because it synchronises the device.  The paper has no
 * counterpart; it is the count of
 * hwc_count through the per-member kernel with its working memory in a fixed
 * device array instead of allocations.
 *  - Calls no cudaMalloc, cudaFree or other allocating routine.  The hash,
 *    statistics and counters live in one file-scope device array of
 *    HWC_NOALLOC_SCRATCH_BYTES (32768 hash slots, about 512 KiB), which every
 *    GPU that loads the library holds until the process exits.
 *  - The job must fit that array: jobs whose histogram could need more than
 *    32768 hash slots (min(count, Hasse-Weil box, number of real Weil
 *    polynomials of degree g for q) above 16384) are rejected
 *    with HWC_ERR_TOO_LARGE before anything runs.
 *  - Families: HWC_FAM_ALL_DEG, HWC_FAM_MONIC_NOSUB and
 *    HWC_FAM_MONIC_NOSUB_SAMPLED (each sample counted for itself); the
 *    reduced and windowed families give HWC_ERR_ARG.
 *  - tables[k-1] (k = 1..g) are handles from hwc_field_tables(q, k), built
 *    beforehand; they are read, not changed.
 *  - Outputs are DEVICE buffers owned by the caller: counts[max_entries*g]
 *    (#C_1..#C_g per entry) and mult[max_entries], in hash order (not
 *    sorted); n_out[3] = number of entries, square-free members, members
 *    examined.  More than max_entries entries gives HWC_ERR_TOO_LARGE.
 *  - The first call on a device sets the library up for it (the device
 *    address of the array, kernel attributes).  Synchronous on `stream`: it
 *    waits to report overflow, so it cannot be called inside a stream
 *    capture.
 *  - Every call shares the one array and clears it first, so calls that
 *    overlap on the GPU (other streams, other host threads) race: run them
 *    one after another. */
#define HWC_NOALLOC_SCRATCH_BYTES (64u + 16u * 32768u)
int hwc_count_noalloc(uint32_t g, uint32_t q, const hwc_family_t *fam, uint64_t first,
                      uint64_t count, const hwc_tables_t *const *tables, uint64_t max_entries,
                      int32_t *counts, uint64_t *mult, uint64_t *n_out, void *stream);

/* ------------------------------------------------------------------ */
/* Measurement                                                         */

/* Rate of dependent, uniformly random 16-bit reads from a shared-memory
 * table of `entries` entries (32..100000), the access pattern Sec. 4 names
 * as the limit of Zech arithmetic on GPUs; `iters` reads per chain, four
 * chains per thread, all SMs.  The denominator of the lookup roofline.
 * Synchronous, current device. */
int hwc_probe_smem_gather(uint32_t entries, uint32_t iters, double *reads_per_s);

#ifdef __cplusplus
}
#endif
#endif /* HWC_H */
