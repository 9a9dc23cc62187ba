// weights.cu -- Berg's multicanonical weight recursion with accumulated error
// weights (Sec. 2.2), one CTA: histogram blocks summed in FP64, the slope
// update per adjacent bin pair, then lnW re-integrated from lnW_0 = 0 by a
// block-wide scan; plus the flatness statistics of Sec. 4.1.
#include "common.cuh"

namespace {

constexpr int kThreads = 1024;

__device__ __forceinline__ double hist_at(const unsigned long long* hist, int n_blocks, int K, int k) {
    unsigned long long s = 0;
    for (int b = 0; b < n_blocks; ++b) s += hist[(int64_t)b * K + k];
    return (double)s;
}

__global__ void __launch_bounds__(kThreads)
berg_kernel(int K, double w, const unsigned long long* __restrict__ hist, int n_blocks, double* lnW,
            double* g_acc, double* beta_out, double* flat_out) {
    extern __shared__ double d[];          // [K - 1] slope differences lnW_k - lnW_{k+1}
    __shared__ double red[32];
    __shared__ double chunk_tot[kThreads];
    const int tid = threadIdx.x;

    // flatness over visited bins
    double n = 0.0, sum = 0.0;
    for (int k = tid; k < K; k += blockDim.x) {
        double h = hist_at(hist, n_blocks, K, k);
        if (h > 0.0) { n += 1.0; sum += h; }
    }
    n = block_sum(n, red);
    sum = block_sum(sum, red);
    const double mean = n > 0.0 ? sum / n : 0.0;
    double var = 0.0, maxdev = 0.0;
    for (int k = tid; k < K; k += blockDim.x) {
        double h = hist_at(hist, n_blocks, K, k);
        if (h > 0.0) {
            var += (h - mean) * (h - mean);
            maxdev = fmax(maxdev, fabs(h - mean) / mean);
        }
    }
    var = block_sum(var, red);
    for (int o = 16; o > 0; o >>= 1) maxdev = fmax(maxdev, __shfl_down_sync(0xffffffffu, maxdev, o));
    __syncthreads();
    if ((tid & 31) == 0) red[tid >> 5] = maxdev;
    __syncthreads();
    if (tid == 0) {
        double mx = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) mx = fmax(mx, red[i]);
        if (flat_out) {
            flat_out[0] = n;
            flat_out[1] = mean;
            flat_out[2] = mean > 0.0 ? sqrt(n > 0.0 ? var / n : 0.0) / mean : 0.0;
            flat_out[3] = mx;
        }
    }
    __syncthreads();

    // slope update: g0 = H_k H_{k+1} / (H_k + H_{k+1}), ghat = g0 / (g_acc + g0)
    for (int k = tid; k + 1 < K; k += blockDim.x) {
        const double h0 = hist_at(hist, n_blocks, K, k), h1 = hist_at(hist, n_blocks, K, k + 1);
        const double g0 = (h0 > 0.0 && h1 > 0.0) ? h0 * h1 / (h0 + h1) : 0.0;
        const double den = g_acc[k] + g0;
        const double ghat = den > 0.0 ? g0 / den : 0.0;
        g_acc[k] = den;
        double dk = lnW[k] - lnW[k + 1];
        if (g0 > 0.0) dk += ghat * (log(h1) - log(h0));
        d[k] = dk;
        if (beta_out) beta_out[k] = dk / w;
    }
    __syncthreads();

    // lnW_0 = 0, lnW_{k+1} = lnW_k - d_k: chunked block scan
    const int M = K - 1;
    const int per = (M + blockDim.x - 1) / blockDim.x;
    const int a = tid * per, b = min(a + per, M);
    double loc = 0.0;
    for (int k = a; k < b; ++k) loc += d[k];
    chunk_tot[tid] = loc;
    __syncthreads();
    if (tid < 32) {   // exclusive scan of the chunk totals by warp 0
        const int per2 = (blockDim.x + 31) / 32;
        double s = 0.0;
        for (int i = tid * per2; i < min((tid + 1) * per2, (int)blockDim.x); ++i) s += chunk_tot[i];
        double incl = s;
        for (int o = 1; o < 32; o <<= 1) {
            double v = __shfl_up_sync(0xffffffffu, incl, o);
            if (tid >= o) incl += v;
        }
        double run = incl - s;
        for (int i = tid * per2; i < min((tid + 1) * per2, (int)blockDim.x); ++i) {
            double v = chunk_tot[i];
            chunk_tot[i] = run;
            run += v;
        }
    }
    __syncthreads();
    double run = chunk_tot[tid];
    if (tid == 0) lnW[0] = 0.0;
    for (int k = a; k < b; ++k) {
        run += d[k];
        lnW[k + 1] = -run;
    }
}

}  // namespace

int phast_launch_berg(int32_t K, double bin_width, const uint64_t* hist, int32_t n_blocks, double* lnW,
                      double* g_acc, double* beta_out, double* flat_out, cudaStream_t st, bool set_attr) {
    size_t sm = sizeof(double) * (size_t)(K > 1 ? K - 1 : 1);
    if (set_attr)   // always the largest K, so that a captured launch never meets a lower limit
        PHAST_CUDA_TRY(cudaFuncSetAttribute(berg_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)(sizeof(double) * (PHAST_MAX_BINS - 1))));
    if (!hist) return PHAST_OK;   // limit only
    berg_kernel<<<1, kThreads, sm, st>>>(K, bin_width, reinterpret_cast<const unsigned long long*>(hist), n_blocks, lnW,
                                         g_acc, beta_out, flat_out);
    PHAST_CUDA_TRY(cudaGetLastError());
    return PHAST_OK;
}

extern "C" int phast_weight_update(int32_t K, double bin_width, const uint64_t* hist, int32_t n_blocks,
                                   double* lnW, double* g_acc, double* beta_out, double* flat_out, void* stream) {
    if (K < 1 || K > PHAST_MAX_BINS) return phast_set_error(PHAST_EINVAL, "phast_weight_update: K %d outside [1, %d]", K, PHAST_MAX_BINS);
    if (!(bin_width > 0.0)) return phast_set_error(PHAST_EINVAL, "phast_weight_update: bin_width must be > 0");
    if (n_blocks < 1) return phast_set_error(PHAST_EINVAL, "phast_weight_update: n_blocks < 1");
    if (!hist || !lnW || (K > 1 && !g_acc)) return phast_set_error(PHAST_EINVAL, "phast_weight_update: NULL argument");
    return phast_launch_berg(K, bin_width, hist, n_blocks, lnW, g_acc, beta_out, flat_out, (cudaStream_t)stream, true);
}
