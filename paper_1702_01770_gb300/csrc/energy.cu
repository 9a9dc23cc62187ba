// energy.cu -- phast_energy (Eq. 2/3 total energy of a batch of
// configurations) and phast_delta_energy (energy change of explicit moves).
// One warp per configuration or move, using the same group machinery as the
// sweep, so these entry points exercise the sweep's own arithmetic.
#include "group.cuh"

namespace {

constexpr int kWarpsPerBlock = 4;

template <typename PT>
__global__ void __launch_bounds__(32 * kWarpsPerBlock)
energy_kernel(const SysDesc d, int B, const double* __restrict__ xyz, double* __restrict__ E_out, SlotLayout L) {
    extern __shared__ __align__(16) unsigned char smem[];
    Group<32> g;
    const int w = threadIdx.x >> 5;
    const int b = blockIdx.x * kWarpsPerBlock + w;
    if (b >= B) return;
    const double* x64 = xyz + (size_t)b * d.N * 3;
    double E;
    if (sizeof(PT) == 8) {
        E = full_energy64<32>(d, x64, g);
    } else {
        Slot<PT> s(smem + (size_t)w * L.bytes, L);
        build_working<32, PT>(d, x64, s, g);
        E = full_energy_working<32, PT>(d, x64, s, g);
        bool out = false;   // a monomer beyond the container's wall: infinite energy
        for (int j = g.lane; j < d.N; j += 32) out |= !inside64(d, ld3(x64 + 3 * j));
        if (__any_sync(g.mask, out)) E = INFINITY;
    }
    if (g.lane == 0) E_out[b] = E;
}

template <typename PT>
__global__ void __launch_bounds__(32 * kWarpsPerBlock)
delta_kernel(const SysDesc d, int B, const double* __restrict__ xyz, const phast_move* __restrict__ moves,
             double* __restrict__ dE_out, double* __restrict__ xyz_new, SlotLayout L) {
    extern __shared__ __align__(16) unsigned char smem[];
    Group<32> g;
    const int w = threadIdx.x >> 5;
    const int b = blockIdx.x * kWarpsPerBlock + w;
    if (b >= B) return;
    const double* x64 = xyz + (size_t)b * d.N * 3;
    Slot<PT> s(smem + (size_t)w * L.bytes, L);
    build_working<32, PT>(d, x64, s, g);
    const phast_move mv = moves[b];
    Proposal P;
    P.type = mv.type; P.chain = mv.chain; P.index = mv.index;
    P.angle = mv.angle; P.uz = P.uw = 0u; P.attempt = -1;
    P.axis = make_double3(mv.axis[0], mv.axis[1], mv.axis[2]);
    P.disp = make_double3(mv.disp[0], mv.disp[1], mv.disp[2]);
    P.angle32 = (float)P.angle;
    P.axis32 = make_float3((float)P.axis.x, (float)P.axis.y, (float)P.axis.z);
    P.disp32 = make_float3((float)P.disp.x, (float)P.disp.y, (float)P.disp.z);
    // a move outside the system (type, chain, interior index, amplitude) is
    // reported as NaN instead of being applied
    bool valid = P.type >= 0 && P.type < PHAST_N_MOVES && P.chain >= 0 && P.chain < d.n_chains;
    if (valid) {
        const int n = d.chain_off[P.chain + 1] - d.chain_off[P.chain];
        if (P.type == PHAST_PIVOT || P.type == PHAST_CRANK) valid = P.index >= 1 && P.index <= n - 2;
        if (P.type == PHAST_BOND) valid = P.index >= 0 && P.index <= n - 2 && isfinite(P.angle);
        else if (P.type == PHAST_CAP) valid = P.index >= 0 && P.index <= n - 1;
        if (P.type == PHAST_TRANS) valid = isfinite(P.disp.x) && isfinite(P.disp.y) && isfinite(P.disp.z);
        else if (P.type != PHAST_BOND) valid = valid && fabs(P.angle) <= PHAST_MAX_ANGLE;
        if (P.type == PHAST_PIVOT || P.type == PHAST_ROT || P.type == PHAST_CAP)
            valid = valid && isfinite(P.axis.x) && isfinite(P.axis.y) && isfinite(P.axis.z);
    }
    if (!valid) P.type = PHAST_TRANS, P.chain = 0, P.index = 0;
    const MoveSet M = move_set(d, P.type, P.chain, P.index);
    double dE = __longlong_as_double(0x7ff8000000000000ll);   // NaN for a degenerate or invalid move
    const bool ok = valid && make_new_positions<32, PT>(d, x64, P, M, s, g);
    const bool wall = ok && !container_ok<32, PT>(d, const_cast<double*>(x64), P, M, s, g, true, 0ull, 0ull, nullptr);
    if (wall) dE = INFINITY;   // beyond the container's wall
    if (ok && !wall) {
        PT fene = (PT)0, tors = (PT)0;
        bool near = false, tnear = false;
        double part = (double)local_delta<32, PT>(d, P, M, s, g, sizeof(PT) == 4 ? &fene : nullptr, &near,
                                                  sizeof(PT) == 4 ? &tors : nullptr, &tnear);
        if constexpr (sizeof(PT) == 4) {
            // a FENE bond near its divergence or a dihedral near degenerate: the exact
            // positions give that kind of term's change
            const bool fx = __ballot_sync(g.mask, near), tx = __ballot_sync(g.mask, tnear);
            if (fx || tx) {
                const double dX = local_delta_exact<32, true>(d, const_cast<double*>(x64), P, M, s, g, true, 0ull,
                                                              0ull, nullptr, fx, tx);
                part += g.lane == 0 ? dX : 0.0;
            }
            if (!fx) part += (double)fene;
            if (!tx) part += (double)tors;
            const DF q = d.box_L > 0.0 ? pair_delta32<32, 3, true>(d, M, P.chain, s, g)
                                       : pair_delta32<32, 3, false>(d, M, P.chain, s, g);
            part += (double)q.hi + (double)q.lo;
        } else {
            part += pair_delta<32, PT, 4>(d, M, P.chain, s, g);
        }
        dE = g.sum(part);
    }
    if (g.lane == 0) dE_out[b] = dE;
    if (xyz_new) {
        if (sizeof(PT) == 4 && valid) prepare_exact<32, PT>(d, x64, P, P.axis, s, g);
        double* out = xyz_new + (size_t)b * d.N * 3;
        for (int j = g.lane; j < d.N; j += 32) {
            double3 y = ld3(x64 + 3 * j);
            if (ok && j >= M.lo && j <= M.hi) y = exact_position(P, s.geo, y);
            out[3 * j + 0] = y.x;
            out[3 * j + 1] = y.y;
            out[3 * j + 2] = y.z;
        }
    }
}

}  // namespace

extern "C" int phast_energy(const phast_system* sys, const phast_ff* ff, int32_t B, const double* xyz,
                            int32_t pair_precision, double* E_out, void* stream) {
    SysDesc d;
    int rc = phast_build_desc(sys, ff, nullptr, &d, "phast_energy");
    if (rc) return rc;
    if (B < 0) return phast_set_error(PHAST_EINVAL, "phast_energy: B < 0");
    if (pair_precision != 32 && pair_precision != 64)
        return phast_set_error(PHAST_EINVAL, "phast_energy: pair_precision must be 32 or 64");
    if (B == 0) return PHAST_OK;
    if (!xyz || !E_out) return phast_set_error(PHAST_EINVAL, "phast_energy: NULL xyz or E_out");
    cudaStream_t st = (cudaStream_t)stream;
    dim3 grid((B + kWarpsPerBlock - 1) / kWarpsPerBlock), block(32 * kWarpsPerBlock);
    if (pair_precision == 64) {
        SlotLayout L = slot_layout<double>(d.N, d.n_chains, d.max_chain);
        energy_kernel<double><<<grid, block, 0, st>>>(d, B, xyz, E_out, L);
    } else {
        SlotLayout L = slot_layout<float>(d.N, d.n_chains, d.max_chain);
        size_t sm = (size_t)L.bytes * kWarpsPerBlock;
        PHAST_CUDA_TRY(cudaFuncSetAttribute(energy_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        energy_kernel<float><<<grid, block, sm, st>>>(d, B, xyz, E_out, L);
    }
    PHAST_CUDA_TRY(cudaGetLastError());
    return PHAST_OK;
}

extern "C" int phast_delta_energy(const phast_system* sys, const phast_ff* ff, int32_t B, const double* xyz,
                                  const phast_move* moves, int32_t pair_precision, double* dE_out,
                                  double* xyz_new_out, void* stream) {
    SysDesc d;
    int rc = phast_build_desc(sys, ff, nullptr, &d, "phast_delta_energy");
    if (rc) return rc;
    if (B < 0) return phast_set_error(PHAST_EINVAL, "phast_delta_energy: B < 0");
    if (pair_precision != 32 && pair_precision != 64)
        return phast_set_error(PHAST_EINVAL, "phast_delta_energy: pair_precision must be 32 or 64");
    if (B == 0) return PHAST_OK;
    if (!xyz || !moves || !dE_out) return phast_set_error(PHAST_EINVAL, "phast_delta_energy: NULL argument");
    cudaStream_t st = (cudaStream_t)stream;
    dim3 grid((B + kWarpsPerBlock - 1) / kWarpsPerBlock), block(32 * kWarpsPerBlock);
    if (pair_precision == 64) {
        SlotLayout L = slot_layout<double>(d.N, d.n_chains, d.max_chain);
        size_t sm = (size_t)L.bytes * kWarpsPerBlock;
        PHAST_CUDA_TRY(cudaFuncSetAttribute(delta_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        delta_kernel<double><<<grid, block, sm, st>>>(d, B, xyz, moves, dE_out, xyz_new_out, L);
    } else {
        SlotLayout L = slot_layout<float>(d.N, d.n_chains, d.max_chain);
        size_t sm = (size_t)L.bytes * kWarpsPerBlock;
        PHAST_CUDA_TRY(cudaFuncSetAttribute(delta_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        delta_kernel<float><<<grid, block, sm, st>>>(d, B, xyz, moves, dE_out, xyz_new_out, L);
    }
    PHAST_CUDA_TRY(cudaGetLastError());
    return PHAST_OK;
}
