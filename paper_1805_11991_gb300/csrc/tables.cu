// tables.cu -- Zech-logarithm tables of F_Q on the device (Sec. 2.3, 3.1-3.2).
//
// F_Q is built as F_p[X]/M(X) with M primitive of degree n = e*k, so X itself
// generates F_Q^x and the antilog table is the walk alpha^i = X^i mod M.  An
// element is the integer sum_t a_t p^t of its coefficients on 1, X, X^2, ...
// The F_q digits of the member index are embedded through a root theta of the
// digit-convention modulus m (first monic irreducible of degree e over F_p):
// digit c = sum_i b_i p^i goes to sum_i b_i theta^i.  Point counts do not
// depend on which root is taken: two embeddings differ by a power of
// Frobenius, which is an automorphism of F_Q carrying points to points.
#include "hwc_internal.cuh"

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <map>
#include <tuple>

namespace hwc {

// ---------------------------------------------------------------------
// host helpers

bool prime_power(uint32_t q, uint32_t *p, uint32_t *e)
{
    if (q < 3 || (q & 1u) == 0) return false;
    uint32_t s = q;
    for (uint32_t d = 3; d * d <= q; d += 2)
        if (q % d == 0) { s = d; break; }
    uint32_t x = q, n = 0;
    while (x % s == 0) { x /= s; ++n; }
    if (x != 1) return false;
    *p = s;
    *e = n;
    return true;
}

namespace {

using Poly = std::vector<uint32_t>;  // coefficients low degree first, mod p

void ptrim(Poly &a)
{
    while (!a.empty() && a.back() == 0) a.pop_back();
}

uint32_t inv_mod(uint32_t a, uint32_t p)
{
    uint64_t r = 1, b = a % p;
    for (uint32_t ex = p - 2; ex; ex >>= 1) {
        if (ex & 1) r = r * b % p;
        b = b * b % p;
    }
    return (uint32_t)r;
}

// a mod b over F_p (b nonzero)
Poly prem(Poly a, const Poly &b, uint32_t p)
{
    ptrim(a);
    uint32_t il = inv_mod(b.back(), p);
    size_t db = b.size() - 1;
    while (a.size() >= b.size()) {
        uint64_t c = (uint64_t)a.back() * il % p;
        size_t sh = a.size() - 1 - db;
        for (size_t i = 0; i <= db; ++i)
            a[sh + i] = (uint32_t)((a[sh + i] + (uint64_t)(p - c) * b[i]) % p);
        ptrim(a);
    }
    return a;
}

Poly pmulmod_h(const Poly &a, const Poly &b, const Poly &f, uint32_t p)
{
    if (a.empty() || b.empty()) return {};
    Poly r(a.size() + b.size() - 1, 0);
    for (size_t i = 0; i < a.size(); ++i)
        for (size_t j = 0; j < b.size(); ++j)
            r[i + j] = (uint32_t)((r[i + j] + (uint64_t)a[i] * b[j]) % p);
    return prem(r, f, p);
}

Poly pgcd(Poly a, Poly b, uint32_t p)
{
    ptrim(a);
    ptrim(b);
    while (!b.empty()) {
        Poly r = prem(a, b, p);
        a = b;
        b = r;
    }
    return a;
}

// Ben-Or: f (monic, degree e) is irreducible over F_p iff
// gcd(f, X^(p^i) - X) = 1 for i = 1 .. e/2.
bool irreducible_ben_or(const Poly &f, uint32_t p)
{
    size_t e = f.size() - 1;
    Poly xp = prem(Poly{0, 1}, f, p);   // X mod f
    for (size_t i = 1; 2 * i <= e; ++i) {
        // xp <- xp^p mod f
        Poly r{1}, b = xp;
        for (uint32_t ex = p; ex; ex >>= 1) {
            if (ex & 1) r = pmulmod_h(r, b, f, p);
            b = pmulmod_h(b, b, f, p);
        }
        xp = r;
        Poly d = xp;
        if (d.size() < 2) d.resize(2, 0);
        d[1] = (d[1] + p - 1) % p;   // X^(p^i) - X
        ptrim(d);
        if (d.empty()) return false;  // f divides X^(p^i) - X
        Poly g = pgcd(f, d, p);
        if (g.size() > 1) return false;
    }
    return true;
}

// digit convention: first monic irreducible of degree e, index sum m_i p^i
bool digit_modulus(uint32_t p, uint32_t e, uint32_t *mq)
{
    uint64_t n = 1;
    for (uint32_t i = 0; i < e; ++i) n *= p;
    for (uint64_t idx = 0; idx < n; ++idx) {
        Poly f(e + 1);
        uint64_t r = idx;
        for (uint32_t i = 0; i < e; ++i) { f[i] = (uint32_t)(r % p); r /= p; }
        f[e] = 1;
        if (irreducible_ben_or(f, p)) {
            for (uint32_t i = 0; i <= e; ++i) mq[i] = f[i];
            return true;
        }
    }
    return false;
}

std::vector<uint32_t> distinct_primes(uint32_t x)
{
    std::vector<uint32_t> out;
    for (uint32_t d = 2; (uint64_t)d * d <= x; ++d)
        if (x % d == 0) {
            out.push_back(d);
            while (x % d == 0) x /= d;
        }
    if (x > 1) out.push_back(x);
    return out;
}

// ---------------------------------------------------------------------
// device polynomial arithmetic over F_p, modulo a monic M of degree n

struct ModPoly {
    uint32_t M[kMaxN + 1];
    uint32_t p;
    int n;
};

__device__ void dmulmod(const uint32_t *a, const uint32_t *b, uint32_t *out, const ModPoly &m)
{
    uint64_t r[2 * kMaxN];
    const int n = m.n;
    const uint32_t p = m.p;
    for (int i = 0; i < 2 * n - 1; ++i) r[i] = 0;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) r[i + j] = (r[i + j] + (uint64_t)a[i] * b[j]) % p;
    for (int t = 2 * n - 2; t >= n; --t) {
        uint64_t c = r[t];
        if (!c) continue;
        for (int i = 0; i < n; ++i) r[t - n + i] = (r[t - n + i] + (p - c) * m.M[i]) % p;
    }
    for (int i = 0; i < n; ++i) out[i] = (uint32_t)r[i];
}

// out = X^ex mod M
__device__ void dpowx(uint64_t ex, uint32_t *out, const ModPoly &m)
{
    uint32_t base[kMaxN], t[kMaxN];
    for (int i = 0; i < m.n; ++i) { base[i] = 0; out[i] = 0; }
    out[0] = 1;
    if (m.n == 1) base[0] = (m.p - m.M[0]) % m.p;   // X = -M_0 mod (X + M_0)
    else base[1] = 1;
    while (ex) {
        if (ex & 1) { dmulmod(out, base, t, m); for (int i = 0; i < m.n; ++i) out[i] = t[i]; }
        ex >>= 1;
        if (ex) { dmulmod(base, base, t, m); for (int i = 0; i < m.n; ++i) base[i] = t[i]; }
    }
}

__device__ bool dis_one(const uint32_t *a, int n)
{
    if (a[0] != 1) return false;
    for (int i = 1; i < n; ++i)
        if (a[i]) return false;
    return true;
}

__device__ uint32_t dpack(const uint32_t *a, int n, uint32_t p)
{
    uint32_t v = 0;
    for (int i = n - 1; i >= 0; --i) v = v * p + a[i];
    return v;
}

struct PrimArgs {
    uint32_t p, L;
    int n, nf;
    uint32_t cof[24];   // L / r for the distinct primes r of L
};

// X has order exactly L in F_p[X]/M  <=>  M is primitive (and irreducible).
__global__ void k_find_primitive(PrimArgs a, uint64_t base, uint64_t count,
                                 unsigned long long *best)
{
    uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= count) return;
    uint64_t idx = base + t;
    ModPoly m;
    m.p = a.p;
    m.n = a.n;
    uint64_t r = idx;
    for (int i = 0; i < a.n; ++i) { m.M[i] = (uint32_t)(r % a.p); r /= a.p; }
    m.M[a.n] = 1;
    if (m.M[0] == 0) return;
    uint32_t v[kMaxN];
    dpowx(a.L, v, m);
    if (!dis_one(v, a.n)) return;
    for (int f = 0; f < a.nf; ++f) {
        dpowx(a.cof[f], v, m);
        if (dis_one(v, a.n)) return;
    }
    atomicMin(best, (unsigned long long)idx);
}

// antilog[i] = X^i, log[X^i] = i; each thread walks a block of B exponents.
__global__ void k_antilog(ModPoly m, uint32_t L, uint32_t B, uint32_t *antilog, uint32_t *logt)
{
    uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    uint64_t start = t * B;
    if (start >= L) return;
    uint32_t cur[kMaxN], x[kMaxN], nxt[kMaxN];
    dpowx(start, cur, m);
    for (int i = 0; i < m.n; ++i) x[i] = 0;
    if (m.n == 1) x[0] = (m.p - m.M[0]) % m.p;
    else x[1] = 1;
    for (uint32_t b = 0; b < B && start + b < L; ++b) {
        uint32_t v = dpack(cur, m.n, m.p);
        antilog[start + b] = v;
        logt[v] = (uint32_t)(start + b);
        dmulmod(cur, x, nxt, m);
        for (int i = 0; i < m.n; ++i) cur[i] = nxt[i];
    }
}

// Z[u] = log(1 + alpha^u) (L if zero), and the layouts the count kernels read:
// doubled over [0, 2L] with poison 2L, tripled over [0, 3L] with poison 3L.
__global__ void k_zech(uint32_t p, uint32_t L, const uint32_t *__restrict__ antilog,
                       const uint32_t *__restrict__ logt, uint32_t *zech, uint16_t *zech2,
                       uint32_t *zech2w, uint16_t *zech3)
{
    const uint64_t top = zech3 ? 3ull * L : 2ull * L;
    for (uint64_t u = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; u <= top;
         u += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t z = L;
        if (u < 3ull * L) {
            const uint32_t um = (uint32_t)(u % L);
            const uint32_t v = antilog[um];
            const uint32_t d0 = v % p;
            const uint32_t w = v - d0 + (d0 + 1 == p ? 0 : d0 + 1);   // v + 1
            z = (w == 0) ? L : logt[w];
        }
        if (u < L) zech[u] = z;
        if (u <= 2ull * L) {
            const uint32_t z2 = (u == 2ull * L || z == L) ? 2 * L : z;
            zech2w[u] = z2;
            if (zech2) zech2[u] = (uint16_t)z2;
        }
        if (zech3) zech3[u] = (uint16_t)((u == 3ull * L || z == L) ? 3 * L : z);
    }
}

// 17-bit layout of the Zech table for fields whose logs need 17 bits: one
// thread per 32 entries writes their low 16 bits and the word of their high
// bits.  Entry L/2 (1 + alpha^(L/2) = 0, Z = L) and entry L carry the marker
// 0x1FFFF, which no log reaches (L < 0x1FFFF).
__global__ void k_zech17(uint32_t L, const uint32_t *__restrict__ zech, uint16_t *lo, uint32_t *hi)
{
    const uint32_t nhi = (L + 32) / 32;
    for (uint32_t w = blockIdx.x * blockDim.x + threadIdx.x; w < nhi; w += gridDim.x * blockDim.x) {
        uint32_t bits = 0;
        for (uint32_t i = 0; i < 32; ++i) {
            const uint32_t n = 32 * w + i;
            if (n > L) break;
            const uint32_t v = (n == L || zech[n] == L) ? 0x1FFFFu : zech[n];
            lo[n] = (uint16_t)(v & 0xFFFFu);
            bits |= (v >> 16) << i;
        }
        hi[w] = bits;
    }
}

// fan-out rows: bit c of row l = [chi(alpha^l + e_c) = -1], e_c the digit c in F_Q;
// alpha^l + e_c = e_c (1 + alpha^(l - log e_c)).  Top bit: alpha^l + e_c = 0 for
// some c (then alpha^l lies in F_q^x).
__global__ void k_rows(uint32_t q, uint32_t L, const uint32_t *__restrict__ zech,
                       const uint32_t *__restrict__ coef_log, uint32_t *rows32,
                       unsigned long long *rows64)
{
    for (uint32_t l = blockIdx.x * blockDim.x + threadIdx.x; l <= L; l += gridDim.x * blockDim.x) {
        if (l == L) {   // y = 0: bit c says chi(e_c) = -1; y + e_0 = 0
            unsigned long long m = 0;
            for (uint32_t c = 1; c < q; ++c)
                if (coef_log[c] & 1u) m |= 1ull << c;
            if (rows32) rows32[L] = (uint32_t)m | 0x80000000u;
            if (rows64) rows64[L] = m | (1ull << 63);
            continue;
        }
        unsigned long long m = l & 1u;   // c = 0: chi(alpha^l) = (-1)^l
        bool zero = false;
        for (uint32_t c = 1; c < q; ++c) {
            const uint32_t lc = coef_log[c];
            const uint32_t n = l >= lc ? l - lc : l + L - lc;
            const uint32_t z = zech[n];
            if (z == L) zero = true;
            else if ((lc + z) & 1u) m |= 1ull << c;
        }
        if (rows32) rows32[l] = (uint32_t)m | (zero ? 0x80000000u : 0u);
        if (rows64) rows64[l] = m | (zero ? (1ull << 63) : 0ull);
    }
}

// zdig[m]: the digit c with alpha^(m s) + e_c = 0, s = L/(q-1); zdig[q-1] = 0
// stands for y = 0 (row index L), where y + e_0 = 0
__global__ void k_zdig(uint32_t q, uint32_t L, const uint32_t *__restrict__ coef_log, uint8_t *zdig)
{
    const uint32_t c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c == 0) zdig[q - 1] = 0;
    if (c == 0 || c >= q) return;
    const uint32_t s = L / (q - 1);
    const uint32_t l = (coef_log[c] + L / 2) % L;   // log(-e_c)
    zdig[l / s] = (uint8_t)c;
}

// digit arithmetic of F_q from its log tables (k = 1): e_a e_b, e_a - e_b, 1/e_a
// as digits, through the inverse of the digit -> log map.
__global__ void k_fq_digit_tables(uint32_t q, uint32_t L, const uint32_t *__restrict__ zech,
                                  const uint32_t *__restrict__ coef_log, uint8_t *mul, uint8_t *sub,
                                  uint8_t *inv)
{
    extern __shared__ uint8_t dig_of_log[];   // [L]
    for (uint32_t c = threadIdx.x; c < q; c += blockDim.x)
        if (c) dig_of_log[coef_log[c]] = (uint8_t)c;
    __syncthreads();
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < q * q; i += gridDim.x * blockDim.x) {
        const uint32_t a = i / q, b = i % q;
        const uint32_t la = coef_log[a], lb = coef_log[b];
        // product
        mul[i] = (a == 0 || b == 0) ? 0 : dig_of_log[(la + lb) % L];
        // difference a - b = a + (-1) b; log(-b) = lb + L/2
        uint8_t d;
        if (b == 0) d = (uint8_t)a;
        else {
            const uint32_t lnb = (lb + L / 2) % L;
            if (a == 0) d = dig_of_log[lnb];
            else {
                // e_a + e_{-b} = e_a (1 + alpha^(lnb - la))
                const uint32_t z = zech[(lnb + L - la) % L];
                d = (z == L) ? 0 : dig_of_log[(la + z) % L];
            }
        }
        sub[i] = d;
        if (b == 0 && a < q) inv[a] = a == 0 ? 0 : dig_of_log[(L - la) % L];
    }
}

// coordinates of F_{q^2} over F_q in the basis {1, alpha}, for alpha^l = e_y0 + e_y1 alpha:
// coord[l] = -y0 | -y1 << 8 | A << 16 | B << 24 with A = 1/y1, B = -y0/y1 when
// y1 != 0, A = 0, B = -y0 when y1 = 0 (digits).  alpha generates F_{q^2}^x, so it
// is not in F_q and every nonzero (y0, y1) names one log:
// e_y0 + e_y1 alpha = e_y0 (1 + alpha^(1 + log e_y1 - log e_y0)) (eq. 2.1).
// Digit arithmetic goes through logs: F_q^x = <alpha^s>, s = L/(q-1).  One block.
__global__ void k_coord2(uint32_t q, uint32_t L, const uint32_t *__restrict__ zech,
                         const uint32_t *__restrict__ coef_log, uint32_t *coord)
{
    __shared__ uint8_t dig[64];   // dig[l / s]: the digit with log l
    const uint32_t s = L / (q - 1), h = L / 2;   // alpha^(L/2) = -1
    for (uint32_t c = threadIdx.x; c < q; c += blockDim.x)
        if (c) dig[coef_log[c] / s] = (uint8_t)c;
    __syncthreads();
    auto digit = [&](uint32_t l) -> uint32_t { return dig[(l % L) / s]; };
    for (uint32_t i = threadIdx.x; i < q * q; i += blockDim.x) {
        const uint32_t y0 = i % q, y1 = i / q;
        if (i == 0) continue;
        const uint32_t l0 = coef_log[y0], l1 = coef_log[y1];
        uint32_t l;
        if (y1 == 0) l = l0;
        else if (y0 == 0) l = (l1 + 1) % L;
        else l = (l0 + zech[(l1 + L - l0 + 1) % L]) % L;   // the Zech value is not L: alpha is not in F_q
        const uint32_t n0 = y0 ? digit(l0 + h) : 0u, n1 = y1 ? digit(l1 + h) : 0u;
        uint32_t A = 0, B = n0;
        if (y1) {
            A = digit(L - l1);
            B = y0 ? digit(l0 + h + L - l1) : 0u;
        }
        coord[l] = n0 | (n1 << 8) | (A << 16) | (B << 24);
    }
}

struct ElemArgs {
    uint32_t p, e, q, n, L;
    uint32_t mq[kMaxE + 1];
};

__device__ void dunpack(uint32_t v, uint32_t *d, uint32_t n, uint32_t p)
{
    for (uint32_t i = 0; i < n; ++i) { d[i] = v % p; v /= p; }
}

// theta = alpha^(s t), s = L/(q-1), t in [0, q-1): smallest t with m(theta) = 0
__global__ void k_theta(ElemArgs a, const uint32_t *__restrict__ antilog, unsigned long long *best)
{
    uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= a.q - 1) return;
    uint64_t th = (uint64_t)(a.L / (a.q - 1)) * t % a.L;
    uint32_t acc[kMaxN] = {}, d[kMaxN];
    for (uint32_t i = 0; i <= a.e; ++i) {
        uint32_t c = a.mq[i];
        if (!c) continue;
        uint32_t pw = antilog[(th * i) % a.L];   // theta^i (theta^0 = antilog[0] = 1)
        dunpack(pw, d, a.n, a.p);
        for (uint32_t j = 0; j < a.n; ++j) acc[j] = (acc[j] + c * d[j]) % a.p;
    }
    for (uint32_t j = 0; j < a.n; ++j)
        if (acc[j]) return;
    atomicMin(best, (unsigned long long)t);
}

// coef_log[c] = log(sum_i b_i theta^i), c = sum_i b_i p^i
__global__ void k_coef_log(ElemArgs a, uint64_t th, const uint32_t *__restrict__ antilog,
                           const uint32_t *__restrict__ logt, uint32_t *coef_log)
{
    uint32_t c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= a.q) return;
    uint32_t acc[kMaxN] = {}, d[kMaxN];
    uint32_t r = c;
    for (uint32_t i = 0; i < a.e; ++i) {
        uint32_t b = r % a.p;
        r /= a.p;
        if (!b) continue;
        uint32_t pw = antilog[(th * i) % a.L];
        dunpack(pw, d, a.n, a.p);
        for (uint32_t j = 0; j < a.n; ++j) acc[j] = (acc[j] + b * d[j]) % a.p;
    }
    uint32_t v = dpack(acc, a.n, a.p);
    coef_log[c] = (v == 0) ? a.L : logt[v];
}

}  // namespace

// ---------------------------------------------------------------------

// Logs j in [0, L) of one element per Frobenius orbit of the elements of F_Q^x
// of exact degree k over F_q (Q = q^k, L = Q - 1): with x = alpha^j the orbit
// of x is {alpha^(j q^i mod L)}, and x has degree m | k over F_q exactly when
// j (q^m - 1) = 0 mod L.  The smallest j of each orbit of size k, ascending.
// Their number is the number of monic irreducible polynomials of degree k over
// F_q.
std::vector<uint32_t> orbit_reps(uint32_t q, uint32_t k, uint32_t L)
{
    std::vector<uint32_t> out;
    uint64_t qm[kMaxG + 1];
    qm[0] = 1;
    for (uint32_t m = 1; m <= k; ++m) qm[m] = qm[m - 1] * q;
    for (uint32_t j = 0; j < L; ++j) {
        bool sub = false;
        for (uint32_t m = 1; m < k && !sub; ++m)
            if (k % m == 0 && (uint64_t)j * (qm[m] - 1) % L == 0) sub = true;
        if (sub) continue;
        bool least = true;
        uint64_t y = j;
        for (uint32_t i = 1; i < k && least; ++i) {
            y = y * q % L;
            if (y < j) least = false;
        }
        if (least) out.push_back(j);
    }
    return out;
}

void tables_destroy(Tables *t)
{
    if (!t) return;
    int cur = -1;
    cudaGetDevice(&cur);
    if (t->device >= 0 && t->device != cur) cudaSetDevice(t->device);
    cudaFree(t->d_antilog);
    cudaFree(t->d_log);
    cudaFree(t->d_zech);
    cudaFree(t->d_coef_log);
    cudaFree(t->d_zech2);
    cudaFree(t->d_zech2w);
    cudaFree(t->d_zech3);
    cudaFree(t->d_z17lo);
    cudaFree(t->d_z17hi);
    cudaFree(t->d_reps);
    cudaFree(t->d_rows32);
    cudaFree(t->d_rows64);
    cudaFree(t->d_zdig);
    cudaFree(t->d_fq_mul);
    cudaFree(t->d_fq_sub);
    cudaFree(t->d_fq_inv);
    cudaFree(t->d_coord2);
    if (t->device >= 0 && t->device != cur && cur >= 0) cudaSetDevice(cur);
    delete t;
}

int tables_build(uint32_t q, uint32_t k, Tables **out, uint64_t max_q)
{
    *out = nullptr;
    uint32_t p, e;
    if (!prime_power(q, &p, &e)) return set_error(HWC_ERR_ARG, "q=%u is not an odd prime power", q);
    if (k < 1 || k > kMaxG) return set_error(HWC_ERR_ARG, "k=%u outside [1,%d]", k, kMaxG);
    uint64_t Q = 1;
    for (uint32_t i = 0; i < k; ++i) Q *= q;
    if (Q > max_q) return set_error(HWC_ERR_TOO_LARGE, "Q=q^k=%llu above %llu", (unsigned long long)Q,
                                    (unsigned long long)max_q);
    if (e > (uint32_t)kMaxE || e * k > (uint32_t)kMaxN)
        return set_error(HWC_ERR_TOO_LARGE, "degree e*k=%u too large", e * k);

    Tables *t = new Tables();
    t->q = q; t->k = k; t->p = p; t->e = e; t->n = e * k;
    t->Q = (uint32_t)Q; t->L = (uint32_t)(Q - 1);
    cudaGetDevice(&t->device);
    const uint32_t L = t->L;
    auto fail = [&](int rc) { tables_destroy(t); return rc; };

    if (!digit_modulus(p, e, t->mq)) return fail(set_error(HWC_ERR_ARG, "no irreducible of degree %u over F_%u", e, p));

    // 1. primitive modulus M: smallest index sum M_i p^i whose X has order L
    PrimArgs pa{};
    pa.p = p; pa.L = L; pa.n = (int)t->n;
    {
        auto pr = distinct_primes(L);
        pa.nf = (int)pr.size();
        for (size_t i = 0; i < pr.size(); ++i) pa.cof[i] = L / pr[i];
    }
    unsigned long long *d_best = nullptr;
    if (cudaMalloc(&d_best, 2 * sizeof(unsigned long long)) != cudaSuccess)
        return fail(set_error(HWC_ERR_NOMEM, "cudaMalloc failed"));
    unsigned long long best = ~0ull;
    const uint64_t ncand = Q;   // p^n candidates
    for (uint64_t base = 0; base < ncand && best == ~0ull; base += 65536) {
        uint64_t cnt = std::min<uint64_t>(65536, ncand - base);
        cudaMemcpy(d_best, &best, sizeof(best), cudaMemcpyHostToDevice);
        k_find_primitive<<<(unsigned)((cnt + 127) / 128), 128>>>(pa, base, cnt, d_best);
        cudaError_t ce = cudaMemcpy(&best, d_best, sizeof(best), cudaMemcpyDeviceToHost);
        if (ce != cudaSuccess) {
            cudaFree(d_best);
            return fail(set_error(HWC_ERR_CUDA, "primitive search: %s", cudaGetErrorString(ce)));
        }
    }
    if (best == ~0ull) {
        cudaFree(d_best);
        return fail(set_error(HWC_ERR_CUDA, "no primitive polynomial found for Q=%u", t->Q));
    }
    ModPoly mp{};
    mp.p = p; mp.n = (int)t->n;
    {
        unsigned long long r = best;
        for (uint32_t i = 0; i < t->n; ++i) { t->M[i] = (uint32_t)(r % p); r /= p; mp.M[i] = t->M[i]; }
        t->M[t->n] = 1; mp.M[t->n] = 1;
    }

    // 2. tables
    bool ok = cudaMalloc(&t->d_antilog, sizeof(uint32_t) * L) == cudaSuccess &&
              cudaMalloc(&t->d_log, sizeof(uint32_t) * t->Q) == cudaSuccess &&
              cudaMalloc(&t->d_zech, sizeof(uint32_t) * L) == cudaSuccess &&
              cudaMalloc(&t->d_coef_log, sizeof(uint32_t) * q) == cudaSuccess &&
              cudaMalloc(&t->d_zech2w, sizeof(uint32_t) * (2ull * L + 1)) == cudaSuccess;
    if (ok && 2ull * L < 65536ull)
        ok = cudaMalloc(&t->d_zech2, sizeof(uint16_t) * (2ull * L + 1)) == cudaSuccess;
    if (ok && 3ull * L < 65536ull)
        ok = cudaMalloc(&t->d_zech3, sizeof(uint16_t) * (3ull * L + 1)) == cudaSuccess;
    const bool z17 = 2ull * L >= 65536ull && L < 0x1FFFFu;
    if (ok && z17)
        ok = cudaMalloc(&t->d_z17lo, sizeof(uint16_t) * (L + 1ull)) == cudaSuccess &&
             cudaMalloc(&t->d_z17hi, sizeof(uint32_t) * ((L + 32ull) / 32)) == cudaSuccess;
    if (!ok) {
        cudaFree(d_best);
        return fail(set_error(HWC_ERR_NOMEM, "cudaMalloc of tables for Q=%u failed", t->Q));
    }
    // log(0) = L (eq. 3.1): the walk writes every nonzero slot
    {
        uint32_t Lh = L;
        cudaMemcpy(t->d_log, &Lh, sizeof(uint32_t), cudaMemcpyHostToDevice);
    }
    const uint32_t B = 64;
    uint64_t nthr = (L + B - 1) / B;
    k_antilog<<<(unsigned)((nthr + 127) / 128), 128>>>(mp, L, B, t->d_antilog, t->d_log);
    k_zech<<<std::max(1u, std::min(4096u, (unsigned)((3ull * L + 256) / 256))), 256>>>(
        p, L, t->d_antilog, t->d_log, t->d_zech, t->d_zech2, t->d_zech2w, t->d_zech3);
    if (z17) k_zech17<<<std::max(1u, std::min(1024u, (L + 32 * 128) / (32 * 128))), 128>>>(L, t->d_zech, t->d_z17lo,
                                                                                           t->d_z17hi);

    // 3. logs of the F_q digits
    ElemArgs ea{};
    ea.p = p; ea.e = e; ea.q = q; ea.n = t->n; ea.L = L;
    for (uint32_t i = 0; i <= e; ++i) ea.mq[i] = t->mq[i];
    uint64_t th = 0;
    if (e > 1) {
        unsigned long long bt = ~0ull;
        cudaMemcpy(d_best, &bt, sizeof(bt), cudaMemcpyHostToDevice);
        k_theta<<<(q + 127) / 128, 128>>>(ea, t->d_antilog, d_best);
        cudaMemcpy(&bt, d_best, sizeof(bt), cudaMemcpyDeviceToHost);
        if (bt == ~0ull) {
            cudaFree(d_best);
            return fail(set_error(HWC_ERR_CUDA, "no root of the digit modulus in F_%u", t->Q));
        }
        th = (uint64_t)(L / (q - 1)) * bt % L;
    }
    k_coef_log<<<(q + 127) / 128, 128>>>(ea, th, t->d_antilog, t->d_log, t->d_coef_log);

    // 4. fan-out rows (digits fit a 64-bit row)
    if (q <= 63) {
        bool rok = cudaMalloc(&t->d_zdig, q) == cudaSuccess;
        if (rok && q <= 31) rok = cudaMalloc(&t->d_rows32, sizeof(uint32_t) * (L + 1)) == cudaSuccess;
        if (rok) rok = cudaMalloc(&t->d_rows64, sizeof(unsigned long long) * (L + 1)) == cudaSuccess;
        if (!rok) {
            cudaFree(d_best);
            return fail(set_error(HWC_ERR_NOMEM, "cudaMalloc of fan-out rows for Q=%u failed", t->Q));
        }
        k_rows<<<std::max(1u, std::min(4096u, (L + 256) / 256)), 256>>>(q, L, t->d_zech, t->d_coef_log,
                                                                         t->d_rows32, t->d_rows64);
        k_zdig<<<1, 64>>>(q, L, t->d_coef_log, t->d_zdig);
        if (k == 1) {
            rok = cudaMalloc(&t->d_fq_mul, q * q) == cudaSuccess && cudaMalloc(&t->d_fq_sub, q * q) == cudaSuccess &&
                  cudaMalloc(&t->d_fq_inv, q) == cudaSuccess;
            if (!rok) {
                cudaFree(d_best);
                return fail(set_error(HWC_ERR_NOMEM, "cudaMalloc of F_%u digit tables failed", q));
            }
            k_fq_digit_tables<<<(q * q + 255) / 256, 256, L>>>(q, L, t->d_zech, t->d_coef_log, t->d_fq_mul,
                                                               t->d_fq_sub, t->d_fq_inv);
        }
        if (k == 2 && q <= 31) {
            if (cudaMalloc(&t->d_coord2, sizeof(uint32_t) * L) != cudaSuccess) {
                cudaFree(d_best);
                return fail(set_error(HWC_ERR_NOMEM, "cudaMalloc of F_%u coordinates failed", t->Q));
            }
            cudaMemset(t->d_coord2, 0, sizeof(uint32_t) * L);   // every entry is written; zero keeps digits in range
            k_coord2<<<1, 256>>>(q, L, t->d_zech, t->d_coef_log, t->d_coord2);
        }
    }
    // 5. one point per Frobenius orbit of the elements of exact degree k
    if (k >= 2) {
        std::vector<uint32_t> reps = orbit_reps(q, k, L);
        t->n_reps = (uint32_t)reps.size();
        if (cudaMalloc(&t->d_reps, sizeof(uint32_t) * reps.size()) != cudaSuccess) {
            cudaFree(d_best);
            return fail(set_error(HWC_ERR_NOMEM, "cudaMalloc of the orbit list of F_%u failed", t->Q));
        }
        cudaMemcpy(t->d_reps, reps.data(), sizeof(uint32_t) * reps.size(), cudaMemcpyHostToDevice);
    }
    cudaError_t ce = cudaDeviceSynchronize();
    cudaFree(d_best);
    if (ce != cudaSuccess) return fail(set_error(HWC_ERR_CUDA, "table kernels: %s", cudaGetErrorString(ce)));
    ce = cudaGetLastError();
    if (ce != cudaSuccess) return fail(set_error(HWC_ERR_CUDA, "table kernels: %s", cudaGetErrorString(ce)));
    *out = t;
    return HWC_OK;
}

int tables_cached(uint32_t q, uint32_t k, const Tables **out, uint64_t max_q)
{
    static std::mutex mu;
    static std::map<std::tuple<int, uint32_t, uint32_t>, Tables *> cache;
    int dev = 0;
    HWC_CUDA_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(mu);
    auto key = std::make_tuple(dev, q, k);
    auto it = cache.find(key);
    if (it != cache.end()) {
        *out = it->second;
        return HWC_OK;
    }
    Tables *t = nullptr;
    int rc = tables_build(q, k, &t, max_q);
    if (rc != HWC_OK) return rc;
    cache[key] = t;
    *out = t;
    return HWC_OK;
}

}  // namespace hwc

// ---------------------------------------------------------------------
// C ABI

extern "C" int hwc_field_tables(uint32_t q, uint32_t k, hwc_tables_t **out)
{
    if (!out) return hwc::set_error(HWC_ERR_ARG, "out is NULL");
    *out = nullptr;
    hwc::Tables *t = nullptr;
    int rc = hwc::tables_build(q, k, &t);
    if (rc != HWC_OK) return rc;
    *out = new hwc_tables{t};
    return HWC_OK;
}

extern "C" int hwc_tables_info(const hwc_tables_t *h, uint32_t *info, uint32_t cap)
{
    if (!h || !h->t || !info) return hwc::set_error(HWC_ERR_ARG, "null argument");
    const hwc::Tables *t = h->t;
    std::vector<uint32_t> v = {t->q, t->k, t->p, t->e, t->Q, t->L, t->n};
    for (uint32_t i = 0; i <= t->n; ++i) v.push_back(t->M[i]);
    for (uint32_t i = 0; i <= t->e; ++i) v.push_back(t->mq[i]);
    if (cap < v.size()) return hwc::set_error(HWC_ERR_ARG, "info needs %zu entries", v.size());
    std::copy(v.begin(), v.end(), info);
    return (int)v.size();
}

extern "C" int hwc_tables_read(const hwc_tables_t *h, uint32_t *antilog, uint32_t *log,
                               uint32_t *zech, uint32_t *coef_log)
{
    if (!h || !h->t) return hwc::set_error(HWC_ERR_ARG, "null tables");
    const hwc::Tables *t = h->t;
    if (antilog) HWC_CUDA_TRY(cudaMemcpy(antilog, t->d_antilog, sizeof(uint32_t) * t->L, cudaMemcpyDeviceToHost));
    if (log) HWC_CUDA_TRY(cudaMemcpy(log, t->d_log, sizeof(uint32_t) * t->Q, cudaMemcpyDeviceToHost));
    if (zech) HWC_CUDA_TRY(cudaMemcpy(zech, t->d_zech, sizeof(uint32_t) * t->L, cudaMemcpyDeviceToHost));
    if (coef_log) HWC_CUDA_TRY(cudaMemcpy(coef_log, t->d_coef_log, sizeof(uint32_t) * t->q, cudaMemcpyDeviceToHost));
    return HWC_OK;
}

extern "C" void hwc_tables_free(hwc_tables_t *h)
{
    if (!h) return;
    hwc::tables_destroy(h->t);
    delete h;
}
