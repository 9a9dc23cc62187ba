// grad.cu -- derivatives of the energy of Eq. 2/3 (with the torsion term) for
// batches of conformations, and multicanonical reweighting of canonical
// averages and their parameter derivatives (Sec. 2.2).
//
// phast_energy_grad: one warp per conformation on the working copy the sweep
// uses (FP32 coordinates relative to chain centroids, or FP64).  Each lane
// owns monomers i = lane, lane + 32, ... and gathers its whole gradient: every
// Lennard-Jones partner j (the pair is evaluated from both ends, no atomics,
// a deterministic order), and the bending and torsion terms that contain i.
// Energies and parameter derivatives count each pair and term once.  Nothing
// is stored between the forward and the backward pass: the backward pass
// recomputes (checkpointed recomputation).
#include "group.cuh"

namespace {

constexpr int kGradWarps = 4;

template <typename PT>
struct V3 {
    PT x, y, z;
};
template <typename PT>
__device__ __forceinline__ V3<PT> sub3(const P4<PT>& a, const P4<PT>& b) {
    return V3<PT>{a.x - b.x, a.y - b.y, a.z - b.z};
}
template <typename PT>
__device__ __forceinline__ PT dot3(const V3<PT>& a, const V3<PT>& b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
template <typename PT>
__device__ __forceinline__ V3<PT> cross3(const V3<PT>& a, const V3<PT>& b) {
    return V3<PT>{a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
template <typename PT>
__device__ __forceinline__ V3<PT> axpy3(PT s, const V3<PT>& a, const V3<PT>& b) {   // s a + b
    return V3<PT>{s * a.x + b.x, s * a.y + b.y, s * a.z + b.z};
}

// d(1 - cos theta_k)/dx_{k-1+which}, theta_k between a = x_k - x_{k-1} and b = x_{k+1} - x_k.
template <typename PT, class Pos>
__device__ V3<PT> bend_grad(const Pos& pos, int o, int k, int which) {
    const P4<PT> x0 = pos(o + k - 1), x1 = pos(o + k), x2 = pos(o + k + 1);
    const V3<PT> a = sub3(x1, x0), b = sub3(x2, x1);
    const PT aa = dot3(a, a), bb = dot3(b, b);
    const PT lab = sqrt(aa) * sqrt(bb);
    const PT cs = dot3(a, b) / lab;
    const V3<PT> dca = axpy3(-cs / aa, a, V3<PT>{b.x / lab, b.y / lab, b.z / lab});   // d cos / d a
    const V3<PT> dcb = axpy3(-cs / bb, b, V3<PT>{a.x / lab, a.y / lab, a.z / lab});   // d cos / d b
    // x_{k-1}: -d cos/d a -> +dca for 1 - cos; x_k: dca - dcb -> -(dca - dcb); x_{k+1}: -dcb
    if (which == 0) return dca;
    if (which == 1) return V3<PT>{dcb.x - dca.x, dcb.y - dca.y, dcb.z - dca.z};
    return V3<PT>{-dcb.x, -dcb.y, -dcb.z};
}

// d cos tau_j / dx_{j+which}: n1 = u x v, n2 = v x w from u, v, w the bonds of monomers j..j+3;
// zero for a degenerate dihedral (|n1|^2 |n2|^2 < 1e-20), where the term is 0.
template <typename PT, class Pos>
__device__ V3<PT> torsion_grad(const Pos& pos, int o, int j, int which) {
    const P4<PT> x0 = pos(o + j), x1 = pos(o + j + 1), x2 = pos(o + j + 2), x3 = pos(o + j + 3);
    const V3<PT> u = sub3(x1, x0), v = sub3(x2, x1), w = sub3(x3, x2);
    const V3<PT> n1 = cross3(u, v), n2 = cross3(v, w);
    const PT n11 = dot3(n1, n1), n22 = dot3(n2, n2);
    if (n11 * n22 < (PT)1e-20) return V3<PT>{0, 0, 0};
    const PT l12 = sqrt(n11) * sqrt(n22);
    const PT cs = dot3(n1, n2) / l12;
    const V3<PT> g1 = axpy3(-cs / n11, n1, V3<PT>{n2.x / l12, n2.y / l12, n2.z / l12});
    const V3<PT> g2 = axpy3(-cs / n22, n2, V3<PT>{n1.x / l12, n1.y / l12, n1.z / l12});
    const V3<PT> du = cross3(v, g1);
    const V3<PT> dv = axpy3((PT)1, cross3(g1, u), cross3(w, g2));
    const V3<PT> dw = cross3(g2, v);
    // u = x1 - x0, v = x2 - x1, w = x3 - x2
    if (which == 0) return V3<PT>{-du.x, -du.y, -du.z};
    if (which == 1) return V3<PT>{du.x - dv.x, du.y - dv.y, du.z - dv.z};
    if (which == 2) return V3<PT>{dv.x - dw.x, dv.y - dw.y, dv.z - dw.z};
    return dw;
}

template <typename PT>
__device__ __forceinline__ PT nearest_count(PT x, PT iL);
template <>
__device__ __forceinline__ float nearest_count<float>(float x, float iL) { return image_count(x, iL); }
template <>
__device__ __forceinline__ double nearest_count<double>(double x, double iL) { return rint(x * iL); }

template <typename PT>
__global__ void __launch_bounds__(32 * kGradWarps)
energy_grad_kernel(const SysDesc d, int B, const double* __restrict__ xyz, double* __restrict__ E_out,
                   double* __restrict__ grad_xyz, double* __restrict__ grad_ff, SlotLayout L) {
    extern __shared__ __align__(16) unsigned char smem[];
    Group<32> g;
    const int w = threadIdx.x >> 5;
    const int b = blockIdx.x * kGradWarps + w;
    if (b >= B) return;
    const double* x64 = xyz + (size_t)b * d.N * 3;
    Slot<PT> s(smem + (size_t)w * L.bytes, L);
    build_working<32, PT>(d, x64, s, g);
    auto pos = [&](int j) -> P4<PT> { return s.r[j]; };
    const FF<PT> f{d};
    const int nc = d.n_chains;
    const PT Lb = f.L(), iLb = f.iL();
    double E = 0.0, gp[5] = {0.0, 0.0, 0.0, 0.0, 0.0};

    // bending and torsion energies, each term once
    for (int c = 0; c < nc; ++c) {
        const int o = d.chain_off[c], n = d.chain_off[c + 1] - o;
        for (int k = 1 + g.lane; k <= n - 2; k += 32) {
            const double t = (double)bend_w<PT>(pos, o, k);
            gp[4] += t;
            E += d.k_bend * t;
        }
        for (int j = g.lane; j <= n - 4; j += 32) {
            const double t = (double)torsion_w<PT>(pos, o, j);
            gp[3] -= t;
            E -= d.k_tors * t;
        }
        if (d.k_fene != 0.0)
            for (int l = g.lane; l <= n - 2; l += 32) E += (double)fene_w<PT>(d, pos, o, l);
    }
    bool out = false;   // a monomer beyond the container's wall: infinite energy
    for (int j = g.lane; j < d.N; j += 32) out |= !inside64(d, ld3(x64 + 3 * j));
    // each lane's monomers: Lennard-Jones partners, then its local terms
    for (int i = g.lane; i < d.N; i += 32) {
        const P4<PT> a = s.r[i];
        const int ci = a.tag >> 1, si = a.tag & 1;
        PT gx = 0, gy = 0, gz = 0;
        PT e_i = 0, p_aa = 0, p_bb = 0, p_ab = 0;
        for (int j = 0; j < d.N; ++j) {
            const P4<PT> q = s.r[j];
            const int cj = q.tag >> 1;
            if (j == i || (ci == cj && (j == i - 1 || j == i + 1))) continue;
            PT dx = a.x - q.x, dy = a.y - q.y, dz = a.z - q.z;
            PT k = f.kin();
            if (ci != cj) {
                const P4<PT> sh = s.D[ci * nc + cj];
                dx += sh.x; dy += sh.y; dz += sh.z;
                if (d.box_L > 0.0) {
                    dx -= Lb * nearest_count<PT>(dx, iLb);
                    dy -= Lb * nearest_count<PT>(dy, iLb);
                    dz -= Lb * nearest_count<PT>(dz, iLb);
                }
                k = f.kout();
            }
            const int sj = q.tag & 1;
            const PT C = f.C(2 * si + sj);
            const PT sv = (PT)1 / (dx * dx + dy * dy + dz * dz);
            const PT s3 = sv * sv * sv, s6 = s3 * s3;
            const PT fr = (PT)2 * k * sv * ((PT)3 * C * s3 - (PT)6 * s6);   // 2 dphi/d(r^2)
            gx += fr * dx;
            gy += fr * dy;
            gz += fr * dz;
            if (i < j) {
                e_i += k * (s6 - C * s3);
                const PT t = k * s3;
                if (si != sj) p_ab -= t;
                else if (si == 0) p_aa -= t;
                else p_bb -= t;
            }
        }
        E += (double)e_i;
        gp[0] += (double)p_aa;
        gp[1] += (double)p_bb;
        gp[2] += (double)p_ab;
        if (grad_xyz) {
            const int o = d.chain_off[ci], n = d.chain_off[ci + 1] - o, li = i - o;
            for (int k = li - 1; k <= li + 1; ++k) {   // bends containing i
                if (k < 1 || k > n - 2) continue;
                const V3<PT> t = bend_grad<PT>(pos, o, k, li - (k - 1));
                gx += f.kbend() * t.x;
                gy += f.kbend() * t.y;
                gz += f.kbend() * t.z;
            }
            for (int j = li - 3; j <= li; ++j) {       // dihedrals containing i: -kappa cos tau
                if (j < 0 || j > n - 4) continue;
                const V3<PT> t = torsion_grad<PT>(pos, o, j, li - j);
                gx -= f.ktors() * t.x;
                gy -= f.ktors() * t.y;
                gz -= f.ktors() * t.z;
            }
            if (d.k_fene != 0.0) {   // bonds of i: d/dr [k R^2 C_F ln(1 - x^2)] = -2 k R C_F x / (1 - x^2)
                for (int l = li - 1; l <= li; ++l) {
                    if (l < 0 || l > n - 2) continue;
                    const V3<PT> b = sub3(s.r[o + l + 1], s.r[o + l]);
                    const PT r = sqrt(dot3(b, b));
                    const PT R = (PT)d.fene_R;
                    const PT x = (r - (PT)d.fene_r0) / R;
                    const PT cf = (PT)d.C_F[2 * d.seq[o + l] + d.seq[o + l + 1]];
                    const PT dphi = (PT)(-2.0 * d.k_fene) * R * cf * x / ((PT)1 - x * x);
                    const PT sg = (l == li) ? (PT)-1 : (PT)1;   // i is the bond's first or second monomer
                    gx += sg * dphi * b.x / r;
                    gy += sg * dphi * b.y / r;
                    gz += sg * dphi * b.z / r;
                }
            }
            double* out = grad_xyz + ((size_t)b * d.N + i) * 3;
            out[0] = (double)gx;
            out[1] = (double)gy;
            out[2] = (double)gz;
        }
    }
    E = g.sum(E);
    if (__any_sync(g.mask, out)) E = INFINITY;
    for (int q = 0; q < 5; ++q) gp[q] = g.sum(gp[q]);
    if (g.lane == 0) {
        if (E_out) E_out[b] = E;
        if (grad_ff)
            for (int q = 0; q < 5; ++q) grad_ff[(size_t)b * 5 + q] = gp[q];
    }
}

// ---------------------------------------------------------------------------
// Reweighting (one CTA per temperature): log-sum-exp maximum, the weighted
// means, then centred moments, all in FP64.
// ---------------------------------------------------------------------------
constexpr int kRwThreads = 512;

__global__ void __launch_bounds__(kRwThreads)
reweight_kernel(int64_t n, const double* __restrict__ E, const double* __restrict__ D, const double* __restrict__ lnW,
                int n_monomers, const double* __restrict__ T, double* E_T, double* cV_T, double* dE_T, double* dcV_T) {
    __shared__ double red[32];
    const int i = blockIdx.x;
    const double beta = 1.0 / T[i];
    double amax = -INFINITY;
    for (int64_t q = threadIdx.x; q < n; q += blockDim.x) amax = fmax(amax, -beta * E[q] - lnW[q]);
    for (int o = 16; o > 0; o >>= 1) amax = fmax(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = amax;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : -INFINITY;
        for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (threadIdx.x == 0) red[0] = v;
    }
    __syncthreads();
    amax = red[0];
    __syncthreads();
    double Z = 0.0, sE = 0.0, sD = 0.0;
    for (int64_t q = threadIdx.x; q < n; q += blockDim.x) {
        const double w = exp(-beta * E[q] - lnW[q] - amax);
        Z += w;
        sE += w * E[q];
        sD += w * D[q];
    }
    Z = block_sum(Z, red);
    sE = block_sum(sE, red);
    sD = block_sum(sD, red);
    const double mE = sE / Z, mD = sD / Z;
    double vE = 0.0, cED = 0.0, m3 = 0.0;
    for (int64_t q = threadIdx.x; q < n; q += blockDim.x) {
        const double w = exp(-beta * E[q] - lnW[q] - amax);
        const double e = E[q] - mE, dd = D[q] - mD;
        vE += w * e * e;
        cED += w * e * dd;
        m3 += w * e * e * dd;
    }
    vE = block_sum(vE, red) / Z;
    cED = block_sum(cED, red) / Z;
    m3 = block_sum(m3, red) / Z;
    if (threadIdx.x == 0) {
        const double nT2 = (double)n_monomers * T[i] * T[i];
        E_T[i] = mE;
        cV_T[i] = vE / nT2;
        dE_T[i] = mD - beta * cED;
        dcV_T[i] = (2.0 * cED - beta * m3) / nT2;
    }
}

}  // namespace

extern "C" int phast_energy_grad(const phast_system* sys, const phast_ff* ff, int32_t B, const double* xyz,
                                 int32_t pair_precision, double* E_out, double* grad_xyz, double* grad_ff,
                                 void* stream) {
    SysDesc d;
    int rc = phast_build_desc(sys, ff, nullptr, &d, "phast_energy_grad");
    if (rc) return rc;
    if (B < 0) return phast_set_error(PHAST_EINVAL, "phast_energy_grad: B < 0");
    if (pair_precision != 32 && pair_precision != 64)
        return phast_set_error(PHAST_EINVAL, "phast_energy_grad: pair_precision must be 32 or 64");
    if (B == 0) return PHAST_OK;
    if (!xyz) return phast_set_error(PHAST_EINVAL, "phast_energy_grad: NULL xyz");
    cudaStream_t st = (cudaStream_t)stream;
    dim3 grid((B + kGradWarps - 1) / kGradWarps), block(32 * kGradWarps);
    if (pair_precision == 64) {
        SlotLayout L = slot_layout<double>(d.N, d.n_chains, d.max_chain);
        size_t sm = (size_t)L.bytes * kGradWarps;
        PHAST_CUDA_TRY(cudaFuncSetAttribute(energy_grad_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        energy_grad_kernel<double><<<grid, block, sm, st>>>(d, B, xyz, E_out, grad_xyz, grad_ff, L);
    } else {
        SlotLayout L = slot_layout<float>(d.N, d.n_chains, d.max_chain);
        size_t sm = (size_t)L.bytes * kGradWarps;
        PHAST_CUDA_TRY(cudaFuncSetAttribute(energy_grad_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        energy_grad_kernel<float><<<grid, block, sm, st>>>(d, B, xyz, E_out, grad_xyz, grad_ff, L);
    }
    PHAST_CUDA_TRY(cudaGetLastError());
    return PHAST_OK;
}

extern "C" int phast_reweight_sensitivity(int64_t n, const double* E, const double* D, const double* lnW,
                                          int32_t n_monomers, int32_t n_T, const double* T, double* E_T,
                                          double* cV_T, double* dE_T, double* dcV_T, void* stream) {
    if (n < 1) return phast_set_error(PHAST_EINVAL, "phast_reweight_sensitivity: n < 1");
    if (n_monomers < 1) return phast_set_error(PHAST_EINVAL, "phast_reweight_sensitivity: n_monomers < 1");
    if (n_T < 0) return phast_set_error(PHAST_EINVAL, "phast_reweight_sensitivity: n_T < 0");
    if (n_T == 0) return PHAST_OK;
    if (!E || !D || !lnW || !T || !E_T || !cV_T || !dE_T || !dcV_T)
        return phast_set_error(PHAST_EINVAL, "phast_reweight_sensitivity: NULL argument");
    reweight_kernel<<<n_T, kRwThreads, 0, (cudaStream_t)stream>>>(n, E, D, lnW, n_monomers, T, E_T, cV_T, dE_T, dcV_T);
    PHAST_CUDA_TRY(cudaGetLastError());
    return PHAST_OK;
}
