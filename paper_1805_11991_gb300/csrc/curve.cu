// curve.cu -- point counts of single curves over large fields (Sec. 4,
// Table 1: one curve y^2 = f(x) of degree 6 counted over F_{p^2}, p up to
// 3001, Q up to 9.0e6).
//
// One curve has too little work per member for the family kernels, so here
// the points of each field are spread over the whole GPU: every warp takes a
// chunk of the field's Frobenius-orbit points and runs the per-member Zech
// chain (field_chi_sum, eq. 2.1) over it with the doubled u32 Zech table read
// from global memory -- 72 MB for F_{3001^2}, resident in the 129 MB L2.
// Per field F_{q^m}, m | k, the warps add sum chi(f(x)) (E_m) and the zeros
// (Z_m) of their chunk into per-curve counters; a last kernel forms
//     #C(F_{q^k}) = q^k + sum_{m | k} m (E_m or N_m - Z_m) + 1 + chi(f(inf))
// (the orbit sums of the family kernels; Sec. 1.1 for the points at infinity).
#include "horner.cuh"

#include <vector>

namespace hwc {
namespace {

struct CurveField {
    uint32_t L, bar, npts, chunk;
    const uint32_t *zech2w;     // doubled u32 Zech table of F_{q^m}
    const uint32_t *coef_log;   // logs of the F_q digits in F_{q^m}
    const uint32_t *pts;        // orbit points of exact degree m (null: every x != 0, m = 1)
    uint32_t m;
};

// E[curve * k + m-1] += sum chi(f(x)), Z[...] += zeros, over this warp's chunk
template <int D>
__global__ void __launch_bounds__(256) k_curve(CurveField F, const uint32_t *__restrict__ coeffs, uint32_t k,
                                              unsigned long long *E, unsigned long long *Z)
{
    const int lane = threadIdx.x & 31;
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t curve = blockIdx.y;
    const uint64_t start = (uint64_t)warp * F.chunk;
    if (start >= F.npts) return;
    const uint32_t cnt = (uint32_t)min((uint64_t)F.chunk, (uint64_t)F.npts - start);
    const uint32_t *cf = coeffs + (uint64_t)curve * (D + 1);
    uint32_t lam[D + 1];
    uint32_t nz = 0;
#pragma unroll
    for (int i = 0; i <= D; ++i) {
        const uint32_t c = cf[i];
        lam[i] = __ldg(F.coef_log + c);
        if (i < D) nz |= (c != 0 ? 1u : 0u) << i;
    }
    int zeros = 0;
    int S = field_chi_sum<D, false>(TabG{F.zech2w}, F.L, F.bar, lam, nz, lane, F.pts ? F.pts + start : nullptr, cnt,
                                    zeros);
    if (F.m == 1 && warp == 0 && lane == 0) {   // x = 0: f(0) = c_0
        if (cf[0] != 0) S += (lam[0] & 1u) ? -1 : 1;
        else zeros += 1;
    }
    S = __reduce_add_sync(kFull, S);
    zeros = __reduce_add_sync(kFull, zeros);
    if (lane == 0) {
        atomicAdd(E + (uint64_t)curve * k + F.m - 1, (unsigned long long)(long long)S);
        atomicAdd(Z + (uint64_t)curve * k + F.m - 1, (unsigned long long)(long long)zeros);
    }
}

// counts[curve] from the per-field sums (N[m-1]: points of field m, x = 0 in m = 1)
__global__ void k_curve_final(uint32_t n, uint32_t k, uint32_t d, uint64_t Q, const uint32_t *__restrict__ coeffs,
                              const uint32_t *__restrict__ coef_log_k, const unsigned long long *E,
                              const unsigned long long *Z, const uint64_t *N, int64_t *counts)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    long long S = 0;
    for (uint32_t m = 1; m <= k; ++m) {
        if (k % m) continue;
        const long long e = (long long)E[(uint64_t)i * k + m - 1];
        const long long z = (long long)Z[(uint64_t)i * k + m - 1];
        S += (long long)m * (((k / m) & 1u) ? e : (long long)N[m - 1] - z);
    }
    long long inf = 1;
    if ((d & 1u) == 0) inf += (coef_log_k[coeffs[(uint64_t)i * (d + 1) + d]] & 1u) ? -1 : 1;
    counts[i] = (int64_t)Q + S + inf;
}

template <int D>
const void *curve_kernel_for() { return (const void *)k_curve<D>; }

const void *curve_kernel(int D)
{
    switch (D) {
    case 3: return curve_kernel_for<3>();
    case 4: return curve_kernel_for<4>();
    case 5: return curve_kernel_for<5>();
    case 6: return curve_kernel_for<6>();
    case 7: return curve_kernel_for<7>();
    case 8: return curve_kernel_for<8>();
    case 9: return curve_kernel_for<9>();
    case 10: return curve_kernel_for<10>();
    default: return nullptr;
    }
}

}  // namespace
}  // namespace hwc

using namespace hwc;

extern "C" int hwc_curve_count(uint32_t q, uint32_t k, uint32_t d, uint64_t n, const uint32_t *coeffs,
                               int64_t *counts, void *stream, float *ms)
{
    uint32_t p = 0, e = 0;
    if (!coeffs || !counts) return set_error(HWC_ERR_ARG, "null argument");
    if (!prime_power(q, &p, &e)) return set_error(HWC_ERR_ARG, "q=%u is not an odd prime power", q);
    if (k < 1 || k > (uint32_t)kMaxG) return set_error(HWC_ERR_ARG, "k=%u outside [1,%d]", k, kMaxG);
    if (d < 3 || d > (uint32_t)kMaxD) return set_error(HWC_ERR_ARG, "degree %u outside [3,%d]", d, kMaxD);
    if (n == 0) return HWC_OK;
    if (n > 65535) return set_error(HWC_ERR_ARG, "at most 65535 curves per call");
    uint64_t Q = 1;
    for (uint32_t i = 0; i < k; ++i) Q *= q;
    if (Q > HWC_MAX_Q_CURVE)
        return set_error(HWC_ERR_TOO_LARGE, "q^k=%llu above %u", (unsigned long long)Q, HWC_MAX_Q_CURVE);
    for (uint64_t i = 0; i < n; ++i) {
        for (uint32_t j = 0; j <= d; ++j)
            if (coeffs[i * (d + 1) + j] >= q) return set_error(HWC_ERR_ARG, "coefficient is not an F_%u digit", q);
        if (coeffs[i * (d + 1) + d] == 0) return set_error(HWC_ERR_ARG, "curve %llu has c_d = 0", (unsigned long long)i);
    }
    const Tables *tab[kMaxG + 1] = {};
    for (uint32_t m = 1; m <= k; ++m) {
        if (k % m) continue;
        int rc = tables_cached(q, m, &tab[m], HWC_MAX_Q_CURVE);
        if (rc) return rc;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const uint64_t ncoef = n * (d + 1);
    // one stream-ordered allocation: coefficients, E, Z, N, counts
    const uint64_t off_e = (ncoef * 4 + 255) / 256 * 256;
    const uint64_t off_z = off_e + (n * k * 8 + 255) / 256 * 256;
    const uint64_t off_n = off_z + (n * k * 8 + 255) / 256 * 256;
    const uint64_t off_c = off_n + 256;
    const uint64_t bytes = off_c + n * 8;
    char *buf = nullptr;
    HWC_CUDA_TRY(cudaMallocAsync((void **)&buf, bytes, s));
    uint32_t *d_coeffs = (uint32_t *)buf;
    unsigned long long *d_E = (unsigned long long *)(buf + off_e), *d_Z = (unsigned long long *)(buf + off_z);
    uint64_t *d_N = (uint64_t *)(buf + off_n);
    int64_t *d_counts = (int64_t *)(buf + off_c);
    uint64_t hN[kMaxG] = {};
    for (uint32_t m = 1; m <= k; ++m)
        if (tab[m]) hN[m - 1] = m == 1 ? q : tab[m]->n_reps;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    int rc = HWC_OK;
    auto cuda = [&](cudaError_t ce, const char *what) {
        if (ce != cudaSuccess && rc == HWC_OK) rc = set_error(HWC_ERR_CUDA, "%s: %s", what, cudaGetErrorString(ce));
    };
    cuda(cudaMemcpyAsync(d_coeffs, coeffs, ncoef * 4, cudaMemcpyHostToDevice, s), "copy coefficients");
    cuda(cudaMemcpyAsync(d_N, hN, sizeof hN, cudaMemcpyHostToDevice, s), "copy point numbers");
    cuda(cudaMemsetAsync(d_E, 0, off_n - off_e, s), "clear sums");
    if (ms) {
        cuda(cudaEventCreate(&ev0), "event");
        cuda(cudaEventCreate(&ev1), "event");
        cuda(cudaEventRecord(ev0, s), "event");
    }
    const int sms = device_sm_count();
    for (uint32_t m = 1; m <= k && rc == HWC_OK; ++m) {
        if (!tab[m]) continue;
        const Tables *t = tab[m];
        CurveField F;
        F.L = t->L;
        F.bar = (uint32_t)((1ull << 32) / t->L);
        F.zech2w = t->d_zech2w;
        F.coef_log = t->d_coef_log;
        F.m = m;
        if (m == 1) {   // F_q: every x != 0, one warp
            F.pts = nullptr;
            F.npts = t->L;
            F.chunk = t->L;
        } else {
            F.pts = t->d_reps;
            F.npts = t->n_reps;
            // about 48 warps of work per SM over all curves, chunks of whole 64-point batches
            const uint64_t want = (uint64_t)sms * 48 / n + 1;
            uint64_t ch = (F.npts + want - 1) / want;
            F.chunk = (uint32_t)std::max<uint64_t>(64, (ch + 63) / 64 * 64);
        }
        const uint64_t warps = (F.npts + F.chunk - 1) / F.chunk;
        dim3 grid((unsigned)((warps + 7) / 8), (unsigned)n);
        void *args[] = {(void *)&F, (void *)&d_coeffs, (void *)&k, (void *)&d_E, (void *)&d_Z};
        cuda(cudaLaunchKernel(curve_kernel((int)d), grid, dim3(256), args, 0, s), "curve kernel");
    }
    if (rc == HWC_OK) {
        k_curve_final<<<(unsigned)((n + 127) / 128), 128, 0, s>>>((uint32_t)n, k, d, Q, d_coeffs,
                                                                   tab[k]->d_coef_log, d_E, d_Z, d_N, d_counts);
        cuda(cudaGetLastError(), "final kernel");
    }
    if (ms) cuda(cudaEventRecord(ev1, s), "event");
    cuda(cudaMemcpyAsync(counts, d_counts, n * 8, cudaMemcpyDeviceToHost, s), "copy counts");
    cudaFreeAsync(buf, s);
    cuda(cudaStreamSynchronize(s), "curve count");
    if (ms && rc == HWC_OK) cuda(cudaEventElapsedTime(ms, ev0, ev1), "event time");
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
    return rc;
}
