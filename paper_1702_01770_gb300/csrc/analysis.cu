// analysis.cu -- microcanonical analysis (Eq. 4-6; ANALYST of Sec. 3.3) with
// canonical reweighting, and error bars either by a jackknife over histogram
// blocks (replicate 0 uses every block; replicate r >= 1 leaves block r-1 out)
// or by binning over iterations (replicate i is iteration i, with its own
// weights and histogram; Sec. 4.1).
//   kernel 1 (one CTA per replicate): S_k, beta_k, C_V,k;
//   kernel 2 (one CTA per replicate and temperature): <E>_T and c_V(T);
//   kernel 3 (one CTA): c_V peak per replicate, values and errors.
#include "common.cuh"

namespace {

constexpr int kThreads = 512;

struct Work {
    double *S, *beta, *CV, *ET, *cVT, *peak;   // [R][K] x3, [R][n_T] x2, [R][2]
};

__host__ __device__ inline size_t work_doubles(int K, int n_T, int R) {
    return (size_t)R * (3 * (size_t)K + 2 * (size_t)n_T + 2);
}

__host__ __device__ inline Work carve(double* base, int K, int n_T, int R) {
    Work w;
    w.S = base;
    w.beta = w.S + (size_t)R * K;
    w.CV = w.beta + (size_t)R * K;
    w.ET = w.CV + (size_t)R * K;
    w.cVT = w.ET + (size_t)R * n_T;
    w.peak = w.cVT + (size_t)R * n_T;
    return w;
}

__device__ __forceinline__ double block_max(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = (blockDim.x + 31) >> 5;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    if (w == 0) {
        v = (l < nw) ? red[l] : -INFINITY;
        for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
        if (l == 0) red[0] = v;
    }
    __syncthreads();
    double r = red[0];
    __syncthreads();
    return r;
}

// H_k of replicate r (block r-1 left out for r >= 1); -1 when no histogram.
__device__ __forceinline__ double rep_hist(const unsigned long long* hist, int n_blocks, int K, int r, int k) {
    if (!hist) return -1.0;
    unsigned long long s = 0;
    for (int b = 0; b < n_blocks; ++b)
        if (b != r - 1) s += hist[(int64_t)b * K + k];
    return (double)s;
}

// iters: replicate r is iteration r (weights row r, histogram row r); else the
// jackknife replicates of the histogram blocks with one weight table.
__global__ void __launch_bounds__(kThreads)
entropy_kernel(int K, double w, const double* __restrict__ lnW, const unsigned long long* __restrict__ hist,
               int n_blocks, int h, Work wk, int iters) {
    __shared__ double red[32];
    const int r = blockIdx.x;
    double* S = wk.S + (size_t)r * K;
    double* beta = wk.beta + (size_t)r * K;
    double* CV = wk.CV + (size_t)r * K;
    const double nan = __longlong_as_double(0x7ff8000000000000ll);
    if (iters) lnW += (size_t)r * K;
    double mx = -INFINITY;
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        double H = iters ? (hist ? (double)hist[(size_t)r * K + k] : -1.0) : rep_hist(hist, n_blocks, K, r, k);
        double s = nan;
        if (H < 0.0) s = -lnW[k];
        else if (H > 0.0) s = -lnW[k] + log(H);
        S[k] = s;
        if (!isnan(s)) mx = fmax(mx, s);
    }
    mx = block_max(mx, red);
    for (int k = threadIdx.x; k < K; k += blockDim.x)
        if (!isnan(S[k])) S[k] -= mx;
    __syncthreads();
    const double he = (double)h * w;
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        double b = nan, cv = nan;
        if (k - h >= 0 && k + h < K && !isnan(S[k - h]) && !isnan(S[k + h])) {
            b = (S[k + h] - S[k - h]) / (2.0 * he);
            if (!isnan(S[k])) {
                double s2 = (S[k + h] - 2.0 * S[k] + S[k - h]) / (he * he);
                cv = -(b * b) / s2;
            }
        }
        beta[k] = b;
        CV[k] = cv;
    }
}

__global__ void __launch_bounds__(256)
canonical_kernel(int K, double e_min, double w, const double* __restrict__ T, int n_T, int n_monomers, Work wk) {
    __shared__ double red[32];
    const int i = blockIdx.x, r = blockIdx.y;
    const double* S = wk.S + (size_t)r * K;
    const double Ti = T[i];
    double lmax = -INFINITY;
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        if (isnan(S[k])) continue;
        double Ek = e_min + ((double)k + 0.5) * w;
        lmax = fmax(lmax, S[k] - Ek / Ti);
    }
    lmax = block_max(lmax, red);
    double Z = 0.0, sE = 0.0;
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        if (isnan(S[k])) continue;
        double Ek = e_min + ((double)k + 0.5) * w;
        double p = exp(S[k] - Ek / Ti - lmax);
        Z += p;
        sE += p * Ek;
    }
    Z = block_sum(Z, red);
    sE = block_sum(sE, red);
    const double mean = sE / Z;
    double var = 0.0;
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        if (isnan(S[k])) continue;
        double Ek = e_min + ((double)k + 0.5) * w;
        double p = exp(S[k] - Ek / Ti - lmax);
        var += p * (Ek - mean) * (Ek - mean);
    }
    var = block_sum(var, red) / Z;
    if (threadIdx.x == 0) {
        wk.ET[(size_t)r * n_T + i] = mean;
        wk.cVT[(size_t)r * n_T + i] = var / ((double)n_monomers * Ti * Ti);
    }
}

__device__ __forceinline__ void jackknife(const double* v, size_t stride, int n, double* val, double* err,
                                          size_t idx) {
    // v[0] full estimate, v[r * stride] leave-block-(r-1)-out replicates
    if (val) val[idx] = v[0];
    if (!err) return;
    if (n < 2) { err[idx] = __longlong_as_double(0x7ff8000000000000ll); return; }
    double m = 0.0;
    for (int r = 1; r <= n; ++r) m += v[r * stride];
    m /= n;
    double s = 0.0;
    for (int r = 1; r <= n; ++r) s += (v[r * stride] - m) * (v[r * stride] - m);
    err[idx] = sqrt((double)(n - 1) / n * s);
}

// Binning over rows 0 .. n_b * block - 1 of v (stride apart), n_b = R / block:
// the mean of the block means and their standard error (NaN for n_b < 2), with
// the oracle's order of summation.
__device__ __forceinline__ void binning(const double* v, size_t stride, int R, int block, double* val, double* err,
                                        size_t idx) {
    const int n_b = R / block;
    double mean = 0.0;
    for (int b = 0; b < n_b; ++b) {
        double s = 0.0;
        for (int i = b * block; i < (b + 1) * block; ++i) s = s + v[(size_t)i * stride];
        mean = mean + s / (double)block;
    }
    mean = mean / (double)n_b;
    if (val) val[idx] = mean;
    if (!err) return;
    if (n_b < 2) { err[idx] = __longlong_as_double(0x7ff8000000000000ll); return; }
    double q = 0.0;
    for (int b = 0; b < n_b; ++b) {
        double s = 0.0;
        for (int i = b * block; i < (b + 1) * block; ++i) s = s + v[(size_t)i * stride];
        const double d = s / (double)block - mean;
        q = q + d * d;
    }
    err[idx] = sqrt(q / ((double)n_b * (double)(n_b - 1)));
}

// block > 0: binning over iterations in blocks of `block`; else the jackknife
// over the n_jk leave-one-block-out replicates.
__global__ void __launch_bounds__(kThreads)
finish_kernel(int K, const double* __restrict__ T, int n_T, int R, int n_jk, Work wk, phast_micro_out o,
              int block) {
    // c_V peak of each replicate: grid maximum, refined by a parabola through it and its neighbours
    for (int r = threadIdx.x; r < R; r += blockDim.x) {
        const double* c = wk.cVT + (size_t)r * n_T;
        double* pk = wk.peak + 2 * (size_t)r;
        if (n_T < 1) { pk[0] = pk[1] = __longlong_as_double(0x7ff8000000000000ll); continue; }
        int im = 0;
        for (int i = 1; i < n_T; ++i) if (c[i] > c[im]) im = i;
        pk[0] = T[im];
        pk[1] = c[im];
        if (im > 0 && im < n_T - 1) {
            double x0 = T[im - 1], x1 = T[im], x2 = T[im + 1], y0 = c[im - 1], y1 = c[im], y2 = c[im + 1];
            double num = (x1 - x0) * (x1 - x0) * (y1 - y2) - (x1 - x2) * (x1 - x2) * (y1 - y0);
            double den = (x1 - x0) * (y1 - y2) - (x1 - x2) * (y1 - y0);
            if (den != 0.0) {
                double xs = x1 - 0.5 * num / den;
                pk[0] = xs;
                pk[1] = y0 * (xs - x1) * (xs - x2) / ((x0 - x1) * (x0 - x2)) +
                        y1 * (xs - x0) * (xs - x2) / ((x1 - x0) * (x1 - x2)) +
                        y2 * (xs - x0) * (xs - x1) / ((x2 - x0) * (x2 - x1));
            }
        }
    }
    __syncthreads();
    if (block > 0) {
        for (int k = threadIdx.x; k < K; k += blockDim.x) {
            binning(wk.S + k, (size_t)K, R, block, o.S, o.S_err, k);
            binning(wk.beta + k, (size_t)K, R, block, o.beta, o.beta_err, k);
            binning(wk.CV + k, (size_t)K, R, block, o.CV, o.CV_err, k);
        }
        for (int i = threadIdx.x; i < n_T; i += blockDim.x) {
            binning(wk.ET + i, (size_t)n_T, R, block, o.E_T, o.E_T_err, i);
            binning(wk.cVT + i, (size_t)n_T, R, block, o.cV_T, o.cV_T_err, i);
        }
        if (threadIdx.x < 2) binning(wk.peak + threadIdx.x, 2, R, block, o.peak, o.peak_err, threadIdx.x);
        return;
    }
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        jackknife(wk.S + k, (size_t)K, n_jk, o.S, o.S_err, k);
        jackknife(wk.beta + k, (size_t)K, n_jk, o.beta, o.beta_err, k);
        jackknife(wk.CV + k, (size_t)K, n_jk, o.CV, o.CV_err, k);
    }
    for (int i = threadIdx.x; i < n_T; i += blockDim.x) {
        jackknife(wk.ET + i, (size_t)n_T, n_jk, o.E_T, o.E_T_err, i);
        jackknife(wk.cVT + i, (size_t)n_T, n_jk, o.cV_T, o.cV_T_err, i);
    }
    if (threadIdx.x < 2) jackknife(wk.peak + threadIdx.x, 2, n_jk, o.peak, o.peak_err, threadIdx.x);
}

// ---------------------------------------------------------------------------
// Free energy (Eq. 7) and the Maxwell construction on the caloric curve
// (ANALYST's Tol_Beta / Tol_L): the equal-area line on beta(E) is the common
// tangent of S(E), an edge of the upper concave hull of (E_k, S_k) over the
// visited bins that spans bins below it.  Among those with a positive slope
// (beta_c = 1/T_c > 0), a latent heat of at least tol_L, and across which
// beta_k = (S_{k+h} - S_{k-h}) / (2 h w) rises by at least tol_beta, the widest
// is taken (the first of equal width).
//
// One CTA per replicate, S in shared memory.  The hull is Andrew's monotone
// chain on one thread with the same FP64 orientation test throughout, so the
// hull vertices are those of the sequential definition even for nearly
// collinear bins; the test of three consecutive bins (k-2, k-1, k), the one
// the chain meets wherever S is concave, is evaluated beforehand by all
// threads, which leaves the serial loop almost free of FP64 instructions.
// The edges, the rise of beta along them, the barrier and f run on all threads.
// ---------------------------------------------------------------------------

// E_k = e_min + (k + 1/2) w, each operation rounded separately.
__device__ __forceinline__ double bin_centre(double e_min, double w, int k) {
    return __dadd_rn(e_min, __dmul_rn(__dadd_rn((double)k, 0.5), w));
}

// Monotone-chain test: drop j (i < j < k) when it lies on or below the chord
// from i to k.
__device__ __forceinline__ bool chain_drops(const double* S, double e_min, double w, int i, int j, int k) {
    const double ei = bin_centre(e_min, w, i), ej = bin_centre(e_min, w, j), ek = bin_centre(e_min, w, k);
    return __dmul_rn(__dsub_rn(S[j], S[i]), __dsub_rn(ek, ei)) <= __dmul_rn(__dsub_rn(S[k], S[i]), __dsub_rn(ej, ei));
}

constexpr size_t kMaxwellSmemPerBin = sizeof(double) + sizeof(int) + 1;   // S, hull, precomputed test

__global__ void __launch_bounds__(kThreads)
maxwell_kernel(int K, double e_min, double w, const double* __restrict__ lnW,
               const unsigned long long* __restrict__ hist, int n_blocks, int h, int n_monomers, double beta_c_in,
               double tol_beta, double tol_L, double* __restrict__ f_out, double* __restrict__ rep) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* S = reinterpret_cast<double*>(smem_raw);                                       // [K]
    int* hull = reinterpret_cast<int*>(smem_raw + sizeof(double) * (size_t)K);             // [K]
    uint8_t* pre = smem_raw + (sizeof(double) + sizeof(int)) * (size_t)K;                  // [K]
    __shared__ double red[32];
    __shared__ int s_nh, s_best_q;
    const int r = blockIdx.x;
    const double nan = __longlong_as_double(0x7ff8000000000000ll);
    const double N = (double)n_monomers;
    double mx = -INFINITY;
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        const double H = rep_hist(hist, n_blocks, K, r, k);
        double s = nan;
        if (H < 0.0) s = -lnW[k];
        else if (H > 0.0) s = -lnW[k] + log(H);
        S[k] = s;
        if (!isnan(s)) mx = fmax(mx, s);
    }
    mx = block_max(mx, red);
    for (int k = threadIdx.x; k < K; k += blockDim.x)
        if (!isnan(S[k])) S[k] -= mx;
    __syncthreads();
    // the chain test of (k-2, k-1, k): 1 drop, 0 keep, 2 not all three visited
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        uint8_t v = 2;
        if (k >= 2 && isfinite(S[k]) && isfinite(S[k - 1]) && isfinite(S[k - 2]))
            v = chain_drops(S, e_min, w, k - 2, k - 1, k) ? 1 : 0;
        pre[k] = v;
    }
    if (threadIdx.x == 0) s_best_q = INT_MAX;
    __syncthreads();
    if (threadIdx.x == 0) {   // upper hull, left to right over the visited bins
        int nh = 0;
        for (int k = 0; k < K; ++k) {
            if (!isfinite(S[k])) continue;
            while (nh >= 2) {
                const int i = hull[nh - 2], j = hull[nh - 1];
                const bool drop = (i == k - 2 && j == k - 1) ? pre[k] == 1 : chain_drops(S, e_min, w, i, j, k);
                if (!drop) break;
                --nh;
            }
            hull[nh++] = k;
        }
        s_nh = nh;
    }
    __syncthreads();
    const int nh = s_nh;
    // qualifying edges, one warp per edge: latent heat, interior bins, the rise
    // max_j (beta_j - min_{k<j} beta_k) over the edge's bins with a defined beta
    double my_L = -1.0;
    int my_q = INT_MAX;
    if (beta_c_in <= 0.0) {
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, n_warps = blockDim.x >> 5;
        const double den = 2.0 * h * w;
        for (int q = warp; q + 1 < nh; q += n_warps) {
            const int a = hull[q], b = hull[q + 1];
            if (b - a < 2) continue;
            bool in = false;
            for (int k = a + 1 + lane; k < b; k += 32) in |= (bool)isfinite(S[k]);
            if (!__any_sync(0xffffffffu, in)) continue;
            const double eab = __dsub_rn(bin_centre(e_min, w, b), bin_centre(e_min, w, a));
            if (!(__ddiv_rn(__dsub_rn(S[b], S[a]), eab) > 0.0)) continue;   // beta_c = 1/T_c > 0
            const double L = __ddiv_rn(eab, N);
            double rise = 0.0, run_min = INFINITY;
            for (int base = a; base <= b; base += 32) {
                const int k = base + lane;
                const bool ok = k <= b && k - h >= 0 && k + h < K && isfinite(S[k - h]) && isfinite(S[k + h]);
                const double bk = ok ? (S[k + h] - S[k - h]) / den : INFINITY;
                double incl = bk;   // inclusive prefix minimum over the lanes
                for (int o = 1; o < 32; o <<= 1) {
                    const double v = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl = fmin(incl, v);
                }
                double excl = __shfl_up_sync(0xffffffffu, incl, 1);
                excl = lane == 0 ? run_min : fmin(run_min, excl);
                if (ok && bk - excl > rise) rise = bk - excl;
                run_min = fmin(run_min, __shfl_sync(0xffffffffu, incl, 31));
            }
            for (int o = 16; o > 0; o >>= 1) rise = fmax(rise, __shfl_xor_sync(0xffffffffu, rise, o));
            if (L >= tol_L && rise >= tol_beta && L > my_L) {   // q rises along this warp's edges
                my_L = L;
                my_q = q;
            }
        }
    }
    const double best_L = block_max(my_L, red);
    if (best_L >= 0.0 && my_L == best_L) atomicMin(&s_best_q, my_q);
    __syncthreads();
    const int best_q = s_best_q;
    double bc = beta_c_in;
    int best_a = -1, best_b = -1;
    if (best_q != INT_MAX) {
        best_a = hull[best_q];
        best_b = hull[best_q + 1];
        bc = __ddiv_rn(__dsub_rn(S[best_b], S[best_a]),
                       __dsub_rn(bin_centre(e_min, w, best_b), bin_centre(e_min, w, best_a)));
    }
    double gap = 0.0;   // the barrier: the largest drop of S below the common tangent
    if (best_a >= 0) {
        const double ea = bin_centre(e_min, w, best_a);
        for (int k = best_a + 1 + threadIdx.x; k < best_b; k += blockDim.x) {
            if (!isfinite(S[k])) continue;
            const double line = __dadd_rn(S[best_a], __dmul_rn(bc, __dsub_rn(bin_centre(e_min, w, k), ea)));
            if (line - S[k] > gap) gap = line - S[k];
        }
    }
    gap = block_max(gap, red);
    if (threadIdx.x == 0) {
        double out[6] = {nan, nan, nan, nan, nan, 0.0};
        if (best_a >= 0) {
            const double ea = bin_centre(e_min, w, best_a), eb = bin_centre(e_min, w, best_b);
            out[0] = bc;
            out[1] = ea / N;
            out[2] = eb / N;
            out[3] = (eb - ea) / N;
            out[4] = gap / __dmul_rn(bc, N);
            out[5] = 1.0;
        } else if (beta_c_in > 0.0) {
            out[0] = beta_c_in;
        }
        for (int q = 0; q < 6; ++q) rep[(size_t)r * 6 + q] = out[q];
    }
    if (r == 0 && f_out) {
        for (int k = threadIdx.x; k < K; k += blockDim.x) {
            const double ek = bin_centre(e_min, w, k);
            f_out[k] = (isfinite(S[k]) && bc > 0.0) ? (ek - S[k] / bc) / N : nan;
        }
    }
}

// Jackknife errors of replicate 0's results over the leave-one-block-out rows;
// NaN when a replicate found no transition; err[5] counts the rows that did.
__global__ void maxwell_err_kernel(int R, const double* __restrict__ rep, double* __restrict__ err) {
    const int q = threadIdx.x;
    if (q >= 6) return;
    const double nan = __longlong_as_double(0x7ff8000000000000ll);
    int found = 0;
    double mean = 0.0;
    for (int r = 1; r <= R; ++r) {
        found += rep[(size_t)r * 6 + 5] != 0.0;
        mean += rep[(size_t)r * 6 + q];
    }
    if (q == 5) { err[5] = (double)found; return; }
    if (R < 2 || found < R) { err[q] = nan; return; }
    mean /= R;
    double ss = 0.0;
    for (int r = 1; r <= R; ++r) {
        const double d = rep[(size_t)r * 6 + q] - mean;
        ss += d * d;
    }
    err[q] = sqrt((double)(R - 1) / R * ss);
}

}  // namespace

extern "C" size_t phast_micro_workspace_size(int32_t K, int32_t n_T, int32_t n_blocks) {
    if (K < 1 || n_T < 0 || n_blocks < 0) return 0;
    int R = 1 + (n_blocks >= 2 ? n_blocks : 0);
    return sizeof(double) * work_doubles(K, n_T, R);
}

extern "C" int phast_micro_analysis(int32_t K, double e_min, double bin_width, const double* lnW, const uint64_t* hist,
                                    int32_t n_blocks, int32_t h, int32_t n_monomers, int32_t n_T, const double* T,
                                    const phast_micro_out* out, void* workspace, size_t workspace_bytes,
                                    void* stream) {
    if (K < 1 || K > PHAST_MAX_BINS) return phast_set_error(PHAST_EINVAL, "phast_micro_analysis: K %d outside [1, %d]", K, PHAST_MAX_BINS);
    if (!(bin_width > 0.0) || !isfinite(e_min)) return phast_set_error(PHAST_EINVAL, "phast_micro_analysis: bad bins");
    if (h < 1 || 2 * h >= K) return phast_set_error(PHAST_EINVAL, "phast_micro_analysis: fd_half_width %d outside [1, K/2)", h);
    if (n_monomers < 1) return phast_set_error(PHAST_EINVAL, "phast_micro_analysis: n_monomers < 1");
    if (n_T < 0 || (n_T > 0 && !T)) return phast_set_error(PHAST_EINVAL, "phast_micro_analysis: bad temperature grid");
    if (!lnW || !out) return phast_set_error(PHAST_EINVAL, "phast_micro_analysis: NULL argument");
    if (hist && n_blocks < 1) return phast_set_error(PHAST_EINVAL, "phast_micro_analysis: n_blocks < 1");
    if (!hist) n_blocks = 0;
    const int R = 1 + (n_blocks >= 2 ? n_blocks : 0);
    const size_t need = sizeof(double) * work_doubles(K, n_T, R);
    if (!workspace || workspace_bytes < need)
        return phast_set_error(PHAST_EINVAL, "phast_micro_analysis: workspace of %zu bytes < %zu", workspace_bytes, need);
    cudaStream_t st = (cudaStream_t)stream;
    Work wk = carve((double*)workspace, K, n_T, R);
    const int njk = n_blocks >= 2 ? n_blocks : 0;
    entropy_kernel<<<R, kThreads, 0, st>>>(K, bin_width, lnW, reinterpret_cast<const unsigned long long*>(hist),
                                           n_blocks, h, wk, 0);
    PHAST_CUDA_TRY(cudaGetLastError());
    if (n_T > 0) {
        canonical_kernel<<<dim3(n_T, R), 256, 0, st>>>(K, e_min, bin_width, T, n_T, n_monomers, wk);
        PHAST_CUDA_TRY(cudaGetLastError());
    }
    finish_kernel<<<1, kThreads, 0, st>>>(K, T, n_T, R, njk, wk, *out, 0);
    PHAST_CUDA_TRY(cudaGetLastError());
    return PHAST_OK;
}

extern "C" size_t phast_micro_binned_workspace_size(int32_t K, int32_t n_T, int32_t n_it) {
    if (K < 1 || n_T < 0 || n_it < 1) return 0;
    return sizeof(double) * work_doubles(K, n_T, n_it);
}

extern "C" int phast_micro_analysis_binned(int32_t K, double e_min, double bin_width, const double* lnW,
                                           const uint64_t* hist, int32_t n_it, int32_t block, int32_t h,
                                           int32_t n_monomers, int32_t n_T, const double* T,
                                           const phast_micro_out* out, void* workspace, size_t workspace_bytes,
                                           void* stream) {
    const char* f = "phast_micro_analysis_binned";
    if (K < 1 || K > PHAST_MAX_BINS) return phast_set_error(PHAST_EINVAL, "%s: K %d outside [1, %d]", f, K, PHAST_MAX_BINS);
    if (!(bin_width > 0.0) || !isfinite(e_min)) return phast_set_error(PHAST_EINVAL, "%s: bad bins", f);
    if (h < 1 || 2 * h >= K) return phast_set_error(PHAST_EINVAL, "%s: fd_half_width %d outside [1, K/2)", f, h);
    if (n_monomers < 1) return phast_set_error(PHAST_EINVAL, "%s: n_monomers < 1", f);
    if (n_T < 0 || (n_T > 0 && !T)) return phast_set_error(PHAST_EINVAL, "%s: bad temperature grid", f);
    if (!lnW || !out) return phast_set_error(PHAST_EINVAL, "%s: NULL argument", f);
    if (n_it < 1 || block < 1 || n_it / block < 1)
        return phast_set_error(PHAST_EINVAL, "%s: %d iterations do not fill one block of %d", f, n_it, block);
    const size_t need = sizeof(double) * work_doubles(K, n_T, n_it);
    if (!workspace || workspace_bytes < need)
        return phast_set_error(PHAST_EINVAL, "%s: workspace of %zu bytes < %zu", f, workspace_bytes, need);
    cudaStream_t st = (cudaStream_t)stream;
    Work wk = carve((double*)workspace, K, n_T, n_it);
    entropy_kernel<<<n_it, kThreads, 0, st>>>(K, bin_width, lnW, reinterpret_cast<const unsigned long long*>(hist),
                                              0, h, wk, 1);
    PHAST_CUDA_TRY(cudaGetLastError());
    if (n_T > 0) {
        canonical_kernel<<<dim3(n_T, n_it), 256, 0, st>>>(K, e_min, bin_width, T, n_T, n_monomers, wk);
        PHAST_CUDA_TRY(cudaGetLastError());
    }
    finish_kernel<<<1, kThreads, 0, st>>>(K, T, n_T, n_it, 0, wk, *out, block);
    PHAST_CUDA_TRY(cudaGetLastError());
    return PHAST_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free variant.  Some callers cannot allocate device memory at the
// point where they need the analysis: a plug-in that runs inside another
// program's CUDA context under a fixed memory budget, or code running between
// the steps of a loop that must not change the device's allocations.  For them
// the workspace lives in a file-scope device array that the library reserves
// when its module is loaded on a device (and keeps until the process exits).
// ---------------------------------------------------------------------------
#include <cuda.h>   // CUcontext and CUresult types only; the driver calls are resolved at run time
#include <mutex>

static __device__ __align__(256) double g_micro_scratch[PHAST_MICRO_NOALLOC_DOUBLES];

namespace {
// The array's name is a host-side stand-in: its device address has to be looked
// up, and it differs between CUDA contexts (a module is loaded once per
// context).  The address is cached per context, keyed by the driver's unique
// context ID, so a context created later (after cudaDeviceReset, or a
// non-primary context a host program makes current) gets its own lookup.
typedef CUresult (*ctx_get_current_fn)(CUcontext*);
typedef CUresult (*ctx_get_id_fn)(CUcontext, unsigned long long*);
struct ScratchEntry {
    unsigned long long ctx_id;
    double* addr;
};
constexpr int kScratchCache = 64;
std::mutex g_scratch_mu;
ScratchEntry g_scratch_cache[kScratchCache];
int g_scratch_used = 0, g_scratch_next = 0;
ctx_get_current_fn g_ctx_get_current = nullptr;
ctx_get_id_fn g_ctx_get_id = nullptr;

// ID of the calling thread's current context; 0 when there is none yet.
int current_ctx_id(unsigned long long* id) {
    *id = 0;
    if (!g_ctx_get_current || !g_ctx_get_id) {
        cudaDriverEntryPointQueryResult q1 = cudaDriverEntryPointSymbolNotFound, q2 = q1;
        void *f1 = nullptr, *f2 = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) != cudaSuccess ||
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) != cudaSuccess ||
            q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2)
            return phast_set_error(PHAST_ECUDA, "phast_micro_analysis_noalloc: driver context queries unavailable");
        g_ctx_get_current = (ctx_get_current_fn)f1;
        g_ctx_get_id = (ctx_get_id_fn)f2;
    }
    CUcontext ctx = nullptr;
    if (g_ctx_get_current(&ctx) != CUDA_SUCCESS)
        return phast_set_error(PHAST_ECUDA, "phast_micro_analysis_noalloc: cuCtxGetCurrent failed");
    if (ctx && g_ctx_get_id(ctx, id) != CUDA_SUCCESS)
        return phast_set_error(PHAST_ECUDA, "phast_micro_analysis_noalloc: cuCtxGetId failed");
    return PHAST_OK;
}
}  // namespace

extern "C" int phast_micro_analysis_noalloc(int32_t K, double e_min, double bin_width, const double* lnW,
                                            const uint64_t* hist, int32_t n_blocks, int32_t h, int32_t n_monomers,
                                            int32_t n_T, const double* T, const phast_micro_out* out, void* stream) {
    if (K < 1 || K > PHAST_MAX_BINS || n_T < 0 || (hist && n_blocks < 1))
        return phast_micro_analysis(K, e_min, bin_width, lnW, hist, n_blocks, h, n_monomers, n_T, T, out,
                                    nullptr, 0, stream);   // reports the argument error
    const int R = 1 + ((hist && n_blocks >= 2) ? n_blocks : 0);
    const size_t need = work_doubles(K, n_T, R);
    if (need > (size_t)PHAST_MICRO_NOALLOC_DOUBLES)
        return phast_set_error(PHAST_EINVAL,
                               "phast_micro_analysis_noalloc: K=%d, n_T=%d, %d blocks need %zu doubles of scratch, "
                               "more than the %d of the static workspace (use phast_micro_analysis)",
                               K, n_T, n_blocks, need, PHAST_MICRO_NOALLOC_DOUBLES);
    double* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_scratch_mu);
        unsigned long long id = 0;
        int rc = current_ctx_id(&id);
        if (rc != PHAST_OK) return rc;
        for (int i = 0; i < g_scratch_used && id; ++i)
            if (g_scratch_cache[i].ctx_id == id) scratch = g_scratch_cache[i].addr;
        if (!scratch) {
            // first call in this context: look the address up (this also makes the
            // runtime's context current when none was)
            void* p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_micro_scratch);
            if (e != cudaSuccess)
                return phast_set_error(PHAST_ECUDA, "phast_micro_analysis_noalloc: cudaGetSymbolAddress: %s",
                                       cudaGetErrorString(e));
            scratch = (double*)p;
            if (!id && (rc = current_ctx_id(&id)) != PHAST_OK) return rc;
            if (id) {
                const int slot = g_scratch_used < kScratchCache ? g_scratch_used++ : (g_scratch_next++ % kScratchCache);
                g_scratch_cache[slot] = ScratchEntry{id, scratch};
            }
        }
    }
    return phast_micro_analysis(K, e_min, bin_width, lnW, hist, n_blocks, h, n_monomers, n_T, T, out, scratch,
                                sizeof(double) * (size_t)PHAST_MICRO_NOALLOC_DOUBLES, stream);
}

extern "C" int phast_maxwell(int32_t K, double e_min, double bin_width, const double* lnW, const uint64_t* hist,
                             int32_t n_blocks, int32_t fd_half_width, int32_t n_monomers, double beta_c,
                             double tol_beta, double tol_L, double* f_out, double* rep, double* err, void* stream) {
    if (K < 1 || K > PHAST_MAX_BINS) return phast_set_error(PHAST_EINVAL, "phast_maxwell: K %d outside [1, %d]", K, PHAST_MAX_BINS);
    if (!(bin_width > 0.0)) return phast_set_error(PHAST_EINVAL, "phast_maxwell: bin_width must be > 0");
    if (!lnW || !rep) return phast_set_error(PHAST_EINVAL, "phast_maxwell: NULL lnW or rep");
    if (hist && n_blocks < 1) return phast_set_error(PHAST_EINVAL, "phast_maxwell: n_blocks < 1");
    if (fd_half_width < 1) return phast_set_error(PHAST_EINVAL, "phast_maxwell: fd_half_width < 1");
    if (n_monomers < 1) return phast_set_error(PHAST_EINVAL, "phast_maxwell: n_monomers < 1");
    if (!(beta_c >= 0.0) || !(tol_beta >= 0.0) || !(tol_L >= 0.0))
        return phast_set_error(PHAST_EINVAL, "phast_maxwell: beta_c, tol_beta, tol_L must be >= 0");
    const int R = (hist && n_blocks >= 2) ? n_blocks : 0;
    const size_t sm = kMaxwellSmemPerBin * (size_t)K;
    cudaStream_t st = (cudaStream_t)stream;
    PHAST_CUDA_TRY(cudaFuncSetAttribute(maxwell_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)(kMaxwellSmemPerBin * PHAST_MAX_BINS)));
    maxwell_kernel<<<1 + R, kThreads, sm, st>>>(K, e_min, bin_width, lnW, reinterpret_cast<const unsigned long long*>(hist),
                                                hist ? n_blocks : 0, fd_half_width, n_monomers, beta_c, tol_beta,
                                                tol_L, f_out, rep);
    PHAST_CUDA_TRY(cudaGetLastError());
    if (err) {
        maxwell_err_kernel<<<1, 32, 0, st>>>(R, rep, err);
        PHAST_CUDA_TRY(cudaGetLastError());
    }
    return PHAST_OK;
}
