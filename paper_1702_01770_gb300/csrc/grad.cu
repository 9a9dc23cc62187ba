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

// The force-field parameters the derivatives are taken in, (C_AA, C_BB, C_AB,
// kappa, kappa_C): from the system's force field, or from a device array of five
// doubles in that order (so a caller holding them on the device needs no copy to
// the host).  c(2 s_i + s_j) is C_LJ of Eq. 1 for letters s_i, s_j.
template <typename PT>
struct Coef {
    PT c0, c1, c2, c3, kt, kb;
    __device__ __forceinline__ PT c(int idx) const { return idx == 0 ? c0 : (idx == 1 ? c1 : (idx == 2 ? c2 : c3)); }
};
template <typename PT>
__device__ __forceinline__ Coef<PT> coef(const SysDesc& d, const double* __restrict__ p) {
    if (p) return Coef<PT>{(PT)p[0], (PT)p[2], (PT)p[2], (PT)p[1], (PT)p[3], (PT)p[4]};
    return Coef<PT>{(PT)d.C[0], (PT)d.C[1], (PT)d.C[2], (PT)d.C[3], (PT)d.k_tors, (PT)d.k_bend};
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
__device__ __forceinline__ double nearest_count<double>(double x, double iL) { return rint(x * iL); }

template <typename PT>
__global__ void __launch_bounds__(32 * kGradWarps)
energy_grad_kernel(const SysDesc d, int B, const double* __restrict__ xyz, double* __restrict__ E_out,
                   double* __restrict__ grad_xyz, double* __restrict__ grad_ff, SlotLayout L,
                   const double* __restrict__ pdev) {
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
    const Coef<PT> cf = coef<PT>(d, pdev);
    const int nc = d.n_chains;
    const PT Lb = f.L(), iLb = f.iL();
    double E = 0.0, gp[5] = {0.0, 0.0, 0.0, 0.0, 0.0};

    // bending and torsion energies, each term once
    for (int c = 0; c < nc; ++c) {
        const int o = d.chain_off[c], n = d.chain_off[c + 1] - o;
        for (int k = 1 + g.lane; k <= n - 2; k += 32) {
            const double t = (double)bend_w<PT>(pos, o, k);
            gp[4] += t;
            E += (double)cf.kb * t;
        }
        for (int j = g.lane; j <= n - 4; j += 32) {
            const double t = (double)torsion_w<PT>(pos, o, j);
            gp[3] -= t;
            E -= (double)cf.kt * t;
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
            const PT C = cf.c(2 * si + sj);
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
                gx += cf.kb * t.x;
                gy += cf.kb * t.y;
                gz += cf.kb * t.z;
            }
            for (int j = li - 3; j <= li; ++j) {       // dihedrals containing i: -kappa cos tau
                if (j < 0 || j > n - 4) continue;
                const V3<PT> t = torsion_grad<PT>(pos, o, j, li - j);
                gx -= cf.kt * t.x;
                gy -= cf.kt * t.y;
                gz -= cf.kt * t.z;
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
// FP32 form: one warp per conformation, each lane the rows i = lane, lane + 32,
// ... of the pair matrix against every partner j, two partners per paired FP32
// instruction (f32x2).  Both ends of a pair are evaluated (each by its own
// row), so every gradient is a plain sum in a fixed order and no atomics are
// needed; energies and parameter derivatives take half of the row sums.  The
// working copy holds FP32 coordinates relative to each chain's origin (its
// centroid rounded to FP32, so the subtraction x - o is exact before the one
// rounding) and the minimum-imaged FP32 differences of the origins.  FP64 is a
// small fraction of FP32 on this chip and every FP64 warp instruction costs its
// full width, so apart from reading the FP64 coordinates and writing the FP64
// gradient the sums run in double-float (two FP32 numbers, TwoSum).
// ---------------------------------------------------------------------------
constexpr int kGrad32Warps = 8;

__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }

template <bool PBC>
__global__ void __launch_bounds__(32 * kGrad32Warps)
energy_grad32_kernel(const SysDesc d, int B, const double* __restrict__ xyz, double* __restrict__ E_out,
                     double* __restrict__ grad_xyz, double* __restrict__ grad_ff, int slot_f4,
                     const double* __restrict__ pdev) {
    extern __shared__ __align__(16) float4 sm4[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int b = blockIdx.x * kGrad32Warps + w;
    if (b >= B) return;
    const unsigned full = 0xffffffffu;
    const int N = d.N, nc = d.n_chains;
    float4* r = sm4 + (size_t)w * slot_f4;            // [N + 1] (x, y, z, tag) relative to the chain origin
    float4* D = r + N + 1;                            // [nc][nc] minimum-imaged origin differences
    float4* org = D + nc * nc;                        // [nc] chain origins (FP32 values)
    const double* x64 = xyz + (size_t)b * N * 3;
    for (int c = 0; c < nc; ++c) {                    // chain centroids in FP32, summed by the warp
        const int o = d.chain_off[c], n = d.chain_off[c + 1] - o;
        float sx = 0.0f, sy = 0.0f, sz = 0.0f;
        for (int j = o + lane; j < o + n; j += 32) {
            sx += (float)x64[3 * j];
            sy += (float)x64[3 * j + 1];
            sz += (float)x64[3 * j + 2];
        }
#pragma unroll
        for (int m = 16; m > 0; m >>= 1) {
            sx += __shfl_xor_sync(full, sx, m);
            sy += __shfl_xor_sync(full, sy, m);
            sz += __shfl_xor_sync(full, sz, m);
        }
        if (lane == 0) org[c] = make_float4(sx / n, sy / n, sz / n, 0.0f);
    }
    __syncwarp();
    for (int j = lane; j < N; j += 32) {
        const int c = d.chain_of[j];
        const float4 oc = org[c];
        r[j] = make_float4((float)(x64[3 * j] - (double)oc.x), (float)(x64[3 * j + 1] - (double)oc.y),
                           (float)(x64[3 * j + 2] - (double)oc.z), __int_as_float((int)d.seq[j] | (c << 1)));
    }
    if (lane == 0) r[N] = make_float4(1.0e4f, 1.0e4f, 1.0e4f, __int_as_float(-2));   // the odd partner slot: far away
    if (nc > 1)
        for (int p = lane; p < nc * nc; p += 32) {
            const int a = p / nc, c = p % nc;
            const float4 oa = org[a], oc = org[c];
            D[p] = make_float4((float)mimage64((double)oa.x - (double)oc.x, d.box_L, d.inv_L),
                               (float)mimage64((double)oa.y - (double)oc.y, d.box_L, d.inv_L),
                               (float)mimage64((double)oa.z - (double)oc.z, d.box_L, d.inv_L), 0.0f);
        }
    __syncwarp();
    auto pos = [&](int j) -> P4<float> {
        const float4 q = r[j];
        P4<float> o;
        o.x = q.x; o.y = q.y; o.z = q.z; o.tag = __float_as_int(q.w);
        return o;
    };
    // the FP64 coordinates, for the dihedrals FP32 cannot resolve (torsion_w)
    auto pos64 = [&](int j) -> double3 { return ld3(x64 + 3 * j); };
    auto pos64p = [&](int j) -> P4<double> {
        P4<double> q;
        q.x = x64[3 * j]; q.y = x64[3 * j + 1]; q.z = x64[3 * j + 2]; q.tag = 0; q.pad = 0;
        return q;
    };
    const FF<float> f{d};
    const Coef<float> cf = coef<float>(d, pdev);
    DF E{0.0f, 0.0f}, gp[5] = {{0.0f, 0.0f}, {0.0f, 0.0f}, {0.0f, 0.0f}, {0.0f, 0.0f}, {0.0f, 0.0f}};
    // bending, torsion and FENE energies, each term once
    for (int c = 0; c < nc; ++c) {
        const int o = d.chain_off[c], n = d.chain_off[c + 1] - o;
        for (int k = 1 + lane; k <= n - 2; k += 32) {
            const float t = bend_w<float>(pos, o, k);
            gp[4] = df_add(gp[4], DF{t, 0.0f});
            E = df_add(E, DF{cf.kb * t, 0.0f});
        }
        for (int j = lane; j <= n - 4; j += 32) {
            bool nr = false;   // a dihedral FP32 cannot resolve: its FP64 value
            float t = torsion_w<float>(pos, o, j, &nr);
            if (nr) t = (float)torsion_term(pos64, o, j);
            gp[3] = df_add(gp[3], DF{-t, 0.0f});
            E = df_add(E, DF{-cf.kt * t, 0.0f});
        }
        if (d.k_fene != 0.0)
            for (int l = lane; l <= n - 2; l += 32) E = df_add(E, DF{fene_w<float>(d, pos, o, l), 0.0f});
    }
    bool out = false;   // a monomer beyond the container's wall: infinite energy
    if (d.sphere_R2 > 0.0)
        for (int j = lane; j < N; j += 32) out |= !inside64(d, ld3(x64 + 3 * j));
    const float2 Mg = f2(12582912.0f), nMg = f2(-12582912.0f);
    const float2 nL = f2(-d.L32), iL = f2(d.iL32);
    for (int i = lane; i < N; i += 32) {
        const float4 a = r[i];
        const int ti = __float_as_int(a.w), ci = ti >> 1, si = ti & 1;
        const float Csame = cf.c(3 * si), Cdiff = cf.c(1);   // partner of the same or the other letter
        float2 gx = f2(0.0f), gy = f2(0.0f), gz = f2(0.0f), e = f2(0.0f), ps = f2(0.0f), pd = f2(0.0f);
        for (int j = 0; j < N; j += 2) {   // partners j, j + 1 (slot N is the far dummy)
            const float4 q0 = r[j], q1 = r[j + 1];
            const int t0 = __float_as_int(q0.w), t1 = __float_as_int(q1.w);
            const int c0 = t0 >> 1, c1 = t1 >> 1;
            // the partner's shift into row i's frame (none within a chain)
            float4 s0 = make_float4(0.f, 0.f, 0.f, 0.f), s1 = s0;
            if (c0 != ci && c0 >= 0) s0 = D[ci * nc + c0];
            if (c1 != ci && c1 >= 0) s1 = D[ci * nc + c1];
            float2 dx = __fadd2_rn(__fadd2_rn(f2(a.x), make_float2(-q0.x, -q1.x)), make_float2(s0.x, s1.x));
            float2 dy = __fadd2_rn(__fadd2_rn(f2(a.y), make_float2(-q0.y, -q1.y)), make_float2(s0.y, s1.y));
            float2 dz = __fadd2_rn(__fadd2_rn(f2(a.z), make_float2(-q0.z, -q1.z)), make_float2(s0.z, s1.z));
            const bool inter0 = c0 != ci && c0 >= 0, inter1 = c1 != ci && c1 >= 0;   // the dummy takes no image
            if (PBC) {   // per-pair minimum image between chains (a zero box length leaves d unchanged)
                const float2 nLp = make_float2(inter0 ? nL.x : 0.0f, inter1 ? nL.y : 0.0f);
                dx = __ffma2_rn(nLp, __fadd2_rn(__ffma2_rn(dx, iL, Mg), nMg), dx);
                dy = __ffma2_rn(nLp, __fadd2_rn(__ffma2_rn(dy, iL, Mg), nMg), dy);
                dz = __ffma2_rn(nLp, __fadd2_rn(__ffma2_rn(dz, iL, Mg), nMg), dz);
            }
            // couplings: 0 for the row itself, its bonded neighbours and the dummy
            const bool x0 = j == i || (!inter0 && (j == i - 1 || j == i + 1)) || t0 < 0;
            const bool x1 = j + 1 == i || (!inter1 && (j + 1 == i - 1 || j + 1 == i + 1)) || t1 < 0;
            const float2 k = make_float2(x0 ? 0.0f : (inter0 ? d.kout32 : d.kin32), x1 ? 0.0f : (inter1 ? d.kout32 : d.kin32));
            const bool same0 = (t0 & 1) == si, same1 = (t1 & 1) == si;
            const float2 C = make_float2(same0 ? Csame : Cdiff, same1 ? Csame : Cdiff);
            float2 r2 = __fmul2_rn(dx, dx);
            r2 = __ffma2_rn(dy, dy, r2);
            r2 = __ffma2_rn(dz, dz, r2);
            r2 = make_float2(x0 ? 1.0e8f : r2.x, x1 ? 1.0e8f : r2.y);   // the row itself has r = 0: keep it finite
            const float2 sv = make_float2(fast_rcp(r2.x), fast_rcp(r2.y));
            const float2 s3 = __fmul2_rn(__fmul2_rn(sv, sv), sv);
            const float2 s6 = __fmul2_rn(s3, s3);
            const float2 ks3 = __fmul2_rn(k, s3);
            // 2 dphi/d(r^2) = 6 k sv (C s3 - 2 s6), phi = k (s6 - C s3)
            const float2 fr = __fmul2_rn(__fmul2_rn(f2(6.0f), __fmul2_rn(k, sv)), __ffma2_rn(C, s3, __fmul2_rn(f2(-2.0f), s6)));
            gx = __ffma2_rn(fr, dx, gx);
            gy = __ffma2_rn(fr, dy, gy);
            gz = __ffma2_rn(fr, dz, gz);
            e = __ffma2_rn(k, __ffma2_rn(__fmul2_rn(f2(-1.0f), C), s3, s6), e);
            ps = __fadd2_rn(ps, make_float2(same0 ? ks3.x : 0.0f, same1 ? ks3.y : 0.0f));
            pd = __fadd2_rn(pd, make_float2(same0 ? 0.0f : ks3.x, same1 ? 0.0f : ks3.y));
        }
        // every pair was taken from both of its ends: halves for the energy and the parameters
        E = df_add(E, df_add(DF{0.5f * e.x, 0.0f}, DF{0.5f * e.y, 0.0f}));
        const DF pss = df_add(DF{-0.5f * ps.x, 0.0f}, DF{-0.5f * ps.y, 0.0f});
        const DF pdd = df_add(DF{-0.5f * pd.x, 0.0f}, DF{-0.5f * pd.y, 0.0f});
        if (si == 0) gp[0] = df_add(gp[0], pss);   // dE/dC_AA (row A, partner A)
        else gp[1] = df_add(gp[1], pss);           // dE/dC_BB
        gp[2] = df_add(gp[2], pdd);                // dE/dC_AB, shared by AB and BA
        if (grad_xyz) {
            float gxs = gx.x + gx.y, gys = gy.x + gy.y, gzs = gz.x + gz.y;
            const int o = d.chain_off[ci], n = d.chain_off[ci + 1] - o, li = i - o;
            for (int kk = li - 1; kk <= li + 1; ++kk) {   // bends containing i
                if (kk < 1 || kk > n - 2) continue;
                const V3<float> t = bend_grad<float>(pos, o, kk, li - (kk - 1));
                gxs += cf.kb * t.x;
                gys += cf.kb * t.y;
                gzs += cf.kb * t.z;
            }
            for (int jj = li - 3; jj <= li; ++jj) {      // dihedrals containing i: -kappa cos tau
                if (jj < 0 || jj > n - 4) continue;
                bool nr = false;
                (void)torsion_w<float>(pos, o, jj, &nr);
                V3<float> t;
                if (nr) {   // FP64, as the value
                    const V3<double> t64 = torsion_grad<double>(pos64p, o, jj, li - jj);
                    t = V3<float>{(float)t64.x, (float)t64.y, (float)t64.z};
                } else {
                    t = torsion_grad<float>(pos, o, jj, li - jj);
                }
                gxs -= cf.kt * t.x;
                gys -= cf.kt * t.y;
                gzs -= cf.kt * t.z;
            }
            if (d.k_fene != 0.0) {   // bonds of i: d/dr [k R^2 C_F ln(1 - x^2)] = -2 k R C_F x / (1 - x^2)
                for (int l = li - 1; l <= li; ++l) {
                    if (l < 0 || l > n - 2) continue;
                    const P4<float> pa = pos(o + l), pb = pos(o + l + 1);
                    const V3<float> bv{pb.x - pa.x, pb.y - pa.y, pb.z - pa.z};
                    const float rb = sqrtf(dot3(bv, bv));
                    const float Rf = (float)d.fene_R;
                    const float xf = (rb - (float)d.fene_r0) / Rf;
                    const float cf = (float)d.C_F[2 * d.seq[o + l] + d.seq[o + l + 1]];
                    const float dphi = (float)(-2.0 * d.k_fene) * Rf * cf * xf / (1.0f - xf * xf);
                    const float sg = (l == li) ? -1.0f : 1.0f;
                    gxs += sg * dphi * bv.x / rb;
                    gys += sg * dphi * bv.y / rb;
                    gzs += sg * dphi * bv.z / rb;
                }
            }
            double* go = grad_xyz + ((size_t)b * N + i) * 3;
            go[0] = (double)gxs;
            go[1] = (double)gys;
            go[2] = (double)gzs;
        }
    }
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) {
        E = df_add(E, DF{__shfl_xor_sync(full, E.hi, m), __shfl_xor_sync(full, E.lo, m)});
#pragma unroll
        for (int q = 0; q < 5; ++q)
            gp[q] = df_add(gp[q], DF{__shfl_xor_sync(full, gp[q].hi, m), __shfl_xor_sync(full, gp[q].lo, m)});
    }
    const bool any_out = __any_sync(full, out);
    if (lane == 0) {
        if (E_out) E_out[b] = any_out ? INFINITY : (double)E.hi + (double)E.lo;
        if (grad_ff)
            for (int q = 0; q < 5; ++q) grad_ff[(size_t)b * 5 + q] = (double)gp[q].hi + (double)gp[q].lo;
    }
}

// Value and gradient of one bending term 1 - cos theta_k at once (FP32, the
// divisions replaced by one reciprocal square root and products): g[0..2] are
// the derivatives with respect to x_{k-1}, x_k, x_{k+1}.
__device__ __forceinline__ float bend_vg(const float4& x0, const float4& x1, const float4& x2, float3 g[3]) {
    const float ax = x1.x - x0.x, ay = x1.y - x0.y, az = x1.z - x0.z;
    const float bx = x2.x - x1.x, by = x2.y - x1.y, bz = x2.z - x1.z;
    const float aa = ax * ax + ay * ay + az * az, bb = bx * bx + by * by + bz * bz;
    const float ab = ax * bx + ay * by + az * bz;
    const float il = rsqrtf(aa * bb);                 // 1 / (|a| |b|)
    const float cs = ab * il;
    const float ia = cs / aa, ib = cs / bb;
    // d cos/d a = b il - cs a / aa, d cos/d b = a il - cs b / bb
    const float3 dca = make_float3(bx * il - ia * ax, by * il - ia * ay, bz * il - ia * az);
    const float3 dcb = make_float3(ax * il - ib * bx, ay * il - ib * by, az * il - ib * bz);
    g[0] = dca;                                                         // x_{k-1}: -(-d cos/d a)
    g[1] = make_float3(dcb.x - dca.x, dcb.y - dca.y, dcb.z - dca.z);   // x_k
    g[2] = make_float3(-dcb.x, -dcb.y, -dcb.z);                        // x_{k+1}
    return 1.0f - cs;
}

// Value and gradient of cos tau_j of monomers j..j+3 at once (FP32); zero for a
// degenerate dihedral (|n1|^2 |n2|^2 < 1e-20), whose term is 0.  A dihedral FP32
// cannot resolve (torsion_unresolved32) is taken in FP64 from x64, the FP64
// coordinates of the chain (monomer j at x64 + 3 j).
__device__ __noinline__ float torsion_vg64(const double* x64, int j, float3 g[4]) {
    auto p = [&](int k) -> P4<double> {
        P4<double> q;
        q.x = x64[3 * k]; q.y = x64[3 * k + 1]; q.z = x64[3 * k + 2]; q.tag = 0; q.pad = 0;
        return q;
    };
    for (int q = 0; q < 4; ++q) {
        const V3<double> t = torsion_grad<double>(p, 0, j, q);
        g[q] = make_float3((float)t.x, (float)t.y, (float)t.z);
    }
    return (float)torsion_term([&](int k) { return ld3(x64 + 3 * k); }, 0, j);
}

__device__ __forceinline__ float torsion_vg(const float4& x0, const float4& x1, const float4& x2, const float4& x3,
                                            float3 g[4], const double* x64, int j) {
    const V3<float> u{x1.x - x0.x, x1.y - x0.y, x1.z - x0.z}, v{x2.x - x1.x, x2.y - x1.y, x2.z - x1.z},
        w{x3.x - x2.x, x3.y - x2.y, x3.z - x2.z};
    const V3<float> n1 = cross3(u, v), n2 = cross3(v, w);
    const float n11 = dot3(n1, n1), n22 = dot3(n2, n2);
    float mx = fmaxf(fmaxf(fabsf(x0.x), fabsf(x0.y)), fabsf(x0.z));
    mx = fmaxf(mx, fmaxf(fmaxf(fabsf(x1.x), fabsf(x1.y)), fabsf(x1.z)));
    mx = fmaxf(mx, fmaxf(fmaxf(fabsf(x2.x), fabsf(x2.y)), fabsf(x2.z)));
    mx = fmaxf(mx, fmaxf(fmaxf(fabsf(x3.x), fabsf(x3.y)), fabsf(x3.z)));
    if (torsion_unresolved32(n11, n22, mx, true)) return torsion_vg64(x64, j, g);
    if (n11 * n22 < 1e-20f) {
        g[0] = g[1] = g[2] = g[3] = make_float3(0.f, 0.f, 0.f);
        return 0.0f;
    }
    const float il = rsqrtf(n11 * n22);
    const float cs = dot3(n1, n2) * il;
    const float c1 = cs / n11, c2 = cs / n22;
    const V3<float> g1{n2.x * il - c1 * n1.x, n2.y * il - c1 * n1.y, n2.z * il - c1 * n1.z};
    const V3<float> g2{n1.x * il - c2 * n2.x, n1.y * il - c2 * n2.y, n1.z * il - c2 * n2.z};
    const V3<float> du = cross3(v, g1);
    const V3<float> dv = axpy3(1.0f, cross3(g1, u), cross3(w, g2));
    const V3<float> dw = cross3(g2, v);
    g[0] = make_float3(-du.x, -du.y, -du.z);
    g[1] = make_float3(du.x - dv.x, du.y - dv.y, du.z - dv.z);
    g[2] = make_float3(dv.x - dw.x, dv.y - dw.y, dv.z - dw.z);
    g[3] = make_float3(dw.x, dw.y, dw.z);
    return cs;
}

__device__ __forceinline__ void acc3(float4* a, int j, float s, float3 g) {
    float4 v = a[j];
    v.x = __fmaf_rn(s, g.x, v.x);
    v.y = __fmaf_rn(s, g.y, v.y);
    v.z = __fmaf_rn(s, g.z, v.z);
    a[j] = v;
}

// The same for one chain in open space (the batch workload of the differentiation
// row): the partners are kept a second time sorted by letter (A monomers, then B,
// each run padded to an even length with a far-away dummy), so the coupling C of
// a run is one value for the row and the parameter sums need no selection; the
// record carries the partner's index, which excludes the row and its bonded
// neighbours.
__global__ void __launch_bounds__(32 * kGrad32Warps)
energy_grad32_chain_kernel(const SysDesc d, int B, const double* __restrict__ xyz, double* __restrict__ E_out,
                           double* __restrict__ grad_xyz, double* __restrict__ grad_ff, int slot_f4,
                           const double* __restrict__ pdev) {
    extern __shared__ __align__(16) float4 sm4[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int b = blockIdx.x * kGrad32Warps + w;
    if (b >= B) return;
    const unsigned full = 0xffffffffu;
    const int N = d.N;
    const int nA = d.n_a_before[N], nB = N - nA;
    const int pA = (nA + 1) & ~1, pB = (nB + 1) & ~1;
    float4* r = sm4 + (size_t)w * slot_f4;   // [N] (x, y, z, tag) relative to the origin, by index
    float4* ps = r + N;                      // [pA + pB] (x, y, z, index): A monomers, then B
    float4* lg = ps + N + 2;                 // [N] gradient of the bending, torsion and FENE terms
    const double* x64 = xyz + (size_t)b * N * 3;
    // origin: the middle monomer rounded to FP32 (an FP32 value, so x - o is exact before
    // its one rounding); FP64 work is kept to the conversions of the coordinates
    const int mid = N / 2;
    const double ox = (double)(float)x64[3 * mid], oy = (double)(float)x64[3 * mid + 1], oz = (double)(float)x64[3 * mid + 2];
    for (int j = lane; j < N; j += 32) {
        const float rx = (float)(x64[3 * j] - ox), ry = (float)(x64[3 * j + 1] - oy), rz = (float)(x64[3 * j + 2] - oz);
        r[j] = make_float4(rx, ry, rz, __int_as_float((int)d.seq[j]));
        lg[j] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        const int ab = d.n_a_before[j];
        ps[d.seq[j] == 0 ? ab : pA + (j - ab)] = make_float4(rx, ry, rz, __int_as_float(j));
    }
    if (lane == 0) {   // the dummies sit far away (their terms underflow to zero)
        if (nA & 1) ps[nA] = make_float4(1.0e4f, 1.0e4f, 1.0e4f, __int_as_float(1 << 20));
        if (nB & 1) ps[pA + nB] = make_float4(1.0e4f, 1.0e4f, 1.0e4f, __int_as_float(1 << 20));
    }
    __syncwarp();
    auto pos = [&](int j) -> P4<float> {
        const float4 q = r[j];
        P4<float> o;
        o.x = q.x; o.y = q.y; o.z = q.z; o.tag = __float_as_int(q.w);
        return o;
    };
    DF E{0.0f, 0.0f}, gp[5] = {{0.0f, 0.0f}, {0.0f, 0.0f}, {0.0f, 0.0f}, {0.0f, 0.0f}, {0.0f, 0.0f}};
    // local terms, each evaluated once with its gradient; terms whose monomers overlap
    // go in different passes (k mod 3 for bends, j mod 4 for dihedrals, l mod 2 for
    // bonds), so a pass adds to disjoint monomers of lg
    const Coef<float> cf = coef<float>(d, pdev);
    const float kb = cf.kb, kt = cf.kt;
    for (int p = 0; p < 3; ++p) {
        for (int k = 1 + p + 3 * lane; k <= N - 2; k += 96) {
            float3 g[3];
            const float t = bend_vg(r[k - 1], r[k], r[k + 1], g);
            gp[4] = df_add(gp[4], DF{t, 0.0f});
            E = df_add(E, DF{kb * t, 0.0f});
            if (grad_xyz)
                for (int q = 0; q < 3; ++q) acc3(lg, k - 1 + q, kb, g[q]);
        }
        __syncwarp();
    }
    for (int p = 0; p < 4; ++p) {
        for (int j = p + 4 * lane; j <= N - 4; j += 128) {
            float3 g[4];
            const float t = torsion_vg(r[j], r[j + 1], r[j + 2], r[j + 3], g, x64, j);
            gp[3] = df_add(gp[3], DF{-t, 0.0f});
            E = df_add(E, DF{-kt * t, 0.0f});
            if (grad_xyz)
                for (int q = 0; q < 4; ++q) acc3(lg, j + q, -kt, g[q]);
        }
        __syncwarp();
    }
    if (d.k_fene != 0.0) {   // bond l: d/dr [k R^2 C_F ln(1 - x^2)] = -2 k R C_F x / (1 - x^2)
        for (int p = 0; p < 2; ++p) {
            for (int l = p + 2 * lane; l <= N - 2; l += 64) {
                E = df_add(E, DF{fene_w<float>(d, pos, 0, l), 0.0f});
                if (!grad_xyz) continue;
                const float4 p0 = r[l], p1 = r[l + 1];
                const float bx = p1.x - p0.x, by = p1.y - p0.y, bz = p1.z - p0.z;
                const float rb = sqrtf(bx * bx + by * by + bz * bz);
                const float Rf = (float)d.fene_R;
                const float xf = (rb - (float)d.fene_r0) / Rf;
                const float cf = (float)d.C_F[2 * d.seq[l] + d.seq[l + 1]];
                const float dphi = (float)(-2.0 * d.k_fene) * Rf * cf * xf / (1.0f - xf * xf);
                const float3 u = make_float3(bx / rb, by / rb, bz / rb);
                acc3(lg, l, -dphi, u);
                acc3(lg, l + 1, dphi, u);
            }
            __syncwarp();
        }
    }
    bool out = false;
    if (d.sphere_R2 > 0.0)
        for (int j = lane; j < N; j += 32) out |= !inside64(d, ld3(x64 + 3 * j));
    const float kin = d.kin32;
    // the local-term gradients of row i, its output and its share of E and the parameters
    auto finish_row = [&](int i, int si, float2 gx, float2 gy, float2 gz, float2 e, float2 prA, float2 prB) {
        // both ends of every pair were taken: halves for the energy and the parameters
        E = df_add(E, df_add(DF{0.5f * e.x, 0.0f}, DF{0.5f * e.y, 0.0f}));
        const DF pa = df_add(DF{-0.5f * prA.x, 0.0f}, DF{-0.5f * prA.y, 0.0f});   // partners A
        const DF pb = df_add(DF{-0.5f * prB.x, 0.0f}, DF{-0.5f * prB.y, 0.0f});   // partners B
        if (si == 0) { gp[0] = df_add(gp[0], pa); gp[2] = df_add(gp[2], pb); }
        else { gp[2] = df_add(gp[2], pa); gp[1] = df_add(gp[1], pb); }
        if (!grad_xyz) return;
        const float4 l4 = lg[i];   // its bending, torsion and FENE terms
        const float gxs = gx.x + gx.y + l4.x, gys = gy.x + gy.y + l4.y, gzs = gz.x + gz.y + l4.z;
        double* go = grad_xyz + ((size_t)b * N + i) * 3;
        go[0] = (double)gxs;
        go[1] = (double)gys;
        go[2] = (double)gzs;
    };
    // two rows per lane at a time, i0 = lane + 64 n and i1 = i0 + 32, against every partner:
    // the partner loads are shared and the two rows' chains are independent
    for (int i0 = lane; i0 < N; i0 += 64) {
        const int i1 = i0 + 32;
        const bool has1 = i1 < N;
        const float4 a0 = r[i0], a1 = has1 ? r[i1] : make_float4(-1.0e4f, -1.0e4f, -1.0e4f, 0.0f);
        const int s0 = __float_as_int(a0.w) & 1, s1 = __float_as_int(a1.w) & 1;
        float2 gx0 = f2(0.0f), gy0 = f2(0.0f), gz0 = f2(0.0f), e0 = f2(0.0f);
        float2 gx1 = f2(0.0f), gy1 = f2(0.0f), gz1 = f2(0.0f), e1 = f2(0.0f);
        float2 pr0[2], pr1[2];
#pragma unroll
        for (int seg = 0; seg < 2; ++seg) {   // partners of letter A, then B: one coupling C per run and row
            const float C0 = cf.c(2 * s0 + seg), C1 = cf.c(2 * s1 + seg);
            const float2 C0v = f2(C0), nC0 = f2(-C0), C1v = f2(C1), nC1 = f2(-C1);
            float2 ap0 = f2(0.0f), ap1 = f2(0.0f);
            const int k0 = seg ? pA : 0, k1 = seg ? pA + pB : pA;
            for (int k = k0; k < k1; k += 2) {
                const float4 q0 = ps[k], q1 = ps[k + 1];
                const int j0 = __float_as_int(q0.w), j1 = __float_as_int(q1.w);
                const float2 qx = make_float2(-q0.x, -q1.x), qy = make_float2(-q0.y, -q1.y),
                             qz = make_float2(-q0.z, -q1.z);
                // row i0
                {
                    const float2 dx = __fadd2_rn(f2(a0.x), qx), dy = __fadd2_rn(f2(a0.y), qy),
                                 dz = __fadd2_rn(f2(a0.z), qz);
                    // the row itself and its bonded neighbours: index within one of i
                    const bool x0 = (unsigned)(j0 - i0 + 1) <= 2u, x1 = (unsigned)(j1 - i0 + 1) <= 2u;
                    float2 r2 = __fmul2_rn(dx, dx);
                    r2 = __ffma2_rn(dy, dy, r2);
                    r2 = __ffma2_rn(dz, dz, r2);
                    r2 = make_float2(x0 ? 1.0e8f : r2.x, x1 ? 1.0e8f : r2.y);
                    const float2 kk = make_float2(x0 ? 0.0f : kin, x1 ? 0.0f : kin);
                    const float2 sv = make_float2(fast_rcp(r2.x), fast_rcp(r2.y));
                    const float2 s3 = __fmul2_rn(__fmul2_rn(sv, sv), sv);
                    const float2 s6 = __fmul2_rn(s3, s3);
                    // 2 dphi/d(r^2) = 6 k sv (C s3 - 2 s6), phi = k (s6 - C s3)
                    const float2 fr = __fmul2_rn(__fmul2_rn(f2(6.0f), __fmul2_rn(kk, sv)),
                                                 __ffma2_rn(C0v, s3, __fmul2_rn(f2(-2.0f), s6)));
                    gx0 = __ffma2_rn(fr, dx, gx0);
                    gy0 = __ffma2_rn(fr, dy, gy0);
                    gz0 = __ffma2_rn(fr, dz, gz0);
                    e0 = __ffma2_rn(kk, __ffma2_rn(nC0, s3, s6), e0);
                    ap0 = __ffma2_rn(kk, s3, ap0);
                }
                // row i1 (a far-away stand-in when it does not exist; its sums are dropped)
                {
                    const float2 dx = __fadd2_rn(f2(a1.x), qx), dy = __fadd2_rn(f2(a1.y), qy),
                                 dz = __fadd2_rn(f2(a1.z), qz);
                    const bool x0 = (unsigned)(j0 - i1 + 1) <= 2u, x1 = (unsigned)(j1 - i1 + 1) <= 2u;
                    float2 r2 = __fmul2_rn(dx, dx);
                    r2 = __ffma2_rn(dy, dy, r2);
                    r2 = __ffma2_rn(dz, dz, r2);
                    r2 = make_float2(x0 ? 1.0e8f : r2.x, x1 ? 1.0e8f : r2.y);
                    const float2 kk = make_float2(x0 ? 0.0f : kin, x1 ? 0.0f : kin);
                    const float2 sv = make_float2(fast_rcp(r2.x), fast_rcp(r2.y));
                    const float2 s3 = __fmul2_rn(__fmul2_rn(sv, sv), sv);
                    const float2 s6 = __fmul2_rn(s3, s3);
                    const float2 fr = __fmul2_rn(__fmul2_rn(f2(6.0f), __fmul2_rn(kk, sv)),
                                                 __ffma2_rn(C1v, s3, __fmul2_rn(f2(-2.0f), s6)));
                    gx1 = __ffma2_rn(fr, dx, gx1);
                    gy1 = __ffma2_rn(fr, dy, gy1);
                    gz1 = __ffma2_rn(fr, dz, gz1);
                    e1 = __ffma2_rn(kk, __ffma2_rn(nC1, s3, s6), e1);
                    ap1 = __ffma2_rn(kk, s3, ap1);
                }
            }
            pr0[seg] = ap0;
            pr1[seg] = ap1;
        }
        finish_row(i0, s0, gx0, gy0, gz0, e0, pr0[0], pr0[1]);
        if (has1) finish_row(i1, s1, gx1, gy1, gz1, e1, pr1[0], pr1[1]);
    }
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) {
        E = df_add(E, DF{__shfl_xor_sync(full, E.hi, m), __shfl_xor_sync(full, E.lo, m)});
#pragma unroll
        for (int q = 0; q < 5; ++q)
            gp[q] = df_add(gp[q], DF{__shfl_xor_sync(full, gp[q].hi, m), __shfl_xor_sync(full, gp[q].lo, m)});
    }
    const bool any_out = __any_sync(full, out);
    // every lane holds the totals: lane 0 converts E, lanes 1..5 the parameter derivatives
    // (one FP64 conversion per lane instead of six on one)
    DF mine = E;
#pragma unroll
    for (int q = 0; q < 5; ++q)
        if (lane == q + 1) mine = gp[q];
    const double v = (double)mine.hi + (double)mine.lo;
    if (lane == 0 && E_out) E_out[b] = any_out ? INFINITY : v;
    if (lane >= 1 && lane <= 5 && grad_ff) grad_ff[(size_t)b * 5 + lane - 1] = v;
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

namespace {
int energy_grad(const phast_system* sys, const phast_ff* ff, int32_t B, const double* xyz, int32_t pair_precision,
                const double* params, double* E_out, double* grad_xyz, double* grad_ff, void* stream) {
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
        energy_grad_kernel<double><<<grid, block, sm, st>>>(d, B, xyz, E_out, grad_xyz, grad_ff, L, params);
    } else if (d.n_chains == 1 && !(d.box_L > 0.0)) {   // per warp: N records, N + 2 sorted partners, N gradients
        const int slot_f4 = 3 * d.N + 2;
        const size_t sm = sizeof(float4) * (size_t)slot_f4 * kGrad32Warps;
        PHAST_CUDA_TRY(cudaFuncSetAttribute(energy_grad32_chain_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        energy_grad32_chain_kernel<<<(B + kGrad32Warps - 1) / kGrad32Warps, 32 * kGrad32Warps, sm, st>>>(
            d, B, xyz, E_out, grad_xyz, grad_ff, slot_f4, params);
    } else {   // per warp: N + 1 records, the nc x nc origin differences, the nc origins
        const int slot_f4 = (d.N + 1) + d.n_chains * d.n_chains + d.n_chains;
        const size_t sm = sizeof(float4) * (size_t)slot_f4 * kGrad32Warps;
        auto fn = d.box_L > 0.0 ? energy_grad32_kernel<true> : energy_grad32_kernel<false>;
        PHAST_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        fn<<<(B + kGrad32Warps - 1) / kGrad32Warps, 32 * kGrad32Warps, sm, st>>>(d, B, xyz, E_out, grad_xyz, grad_ff,
                                                                               slot_f4, params);
    }
    PHAST_CUDA_TRY(cudaGetLastError());
    return PHAST_OK;
}
}  // namespace

extern "C" int phast_energy_grad(const phast_system* sys, const phast_ff* ff, int32_t B, const double* xyz,
                                 int32_t pair_precision, double* E_out, double* grad_xyz, double* grad_ff,
                                 void* stream) {
    return energy_grad(sys, ff, B, xyz, pair_precision, nullptr, E_out, grad_xyz, grad_ff, stream);
}

extern "C" int phast_energy_grad_params(const phast_system* sys, const phast_ff* ff, int32_t B, const double* xyz,
                                        int32_t pair_precision, const double* params, double* E_out,
                                        double* grad_xyz, double* grad_ff, void* stream) {
    if (!params) return phast_set_error(PHAST_EINVAL, "phast_energy_grad_params: NULL params");
    return energy_grad(sys, ff, B, xyz, pair_precision, params, E_out, grad_xyz, grad_ff, stream);
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
